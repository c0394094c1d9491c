// Kernels for K = 3 fibers per voxel.
#define PRISM_K 3
#include "prism_kset.cuh"
