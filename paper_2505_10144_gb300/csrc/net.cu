// periphery network kernels (filled in below)
#include "common.cuh"
