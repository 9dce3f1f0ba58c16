// D2Q9 instantiation of the step kernels (see elbm_kernels.cuh).
#define ELBM_DIM 2
#define ELBM_SUFFIX d2q9
#include "elbm_kernels.cuh"
