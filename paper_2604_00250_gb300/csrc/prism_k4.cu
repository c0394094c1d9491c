// Kernels for K = 4 fibers per voxel.
#define PRISM_K 4
#include "prism_kset.cuh"
