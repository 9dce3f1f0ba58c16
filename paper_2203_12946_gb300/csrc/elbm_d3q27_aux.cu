// D3Q27 instantiation of the companion kernels (see elbm_kernels.cuh): every launcher but
// the step's (elbm_d3q27.cu).
#define ELBM_DIM 3
#define ELBM_SUFFIX d3q27
#define ELBM_PART 2
#include "elbm_kernels.cuh"
