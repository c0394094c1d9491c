// Kernels for K = 2 fibers per voxel.
#define PRISM_K 2
#include "prism_kset.cuh"
