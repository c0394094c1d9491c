// Kernels for K = 5 fibers per voxel.
#define PRISM_K 5
#include "prism_kset.cuh"
