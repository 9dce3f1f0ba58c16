// D3Q27 instantiation of the step kernels (see elbm_kernels.cuh).
#define ELBM_DIM 3
#define ELBM_SUFFIX d3q27
#include "elbm_kernels.cuh"
