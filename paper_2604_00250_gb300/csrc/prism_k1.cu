// Kernels for K = 1 fibers per voxel.
#define PRISM_K 1
#include "prism_kset.cuh"
