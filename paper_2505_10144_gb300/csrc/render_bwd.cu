// backward kernels (filled in below)
#include "common.cuh"
