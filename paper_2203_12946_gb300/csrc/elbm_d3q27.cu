// D3Q27 instantiation of the step kernels (see elbm_kernels.cuh): the step launcher;
// elbm_d3q27_aux.cu holds the other launchers, so the two compile in parallel.
#define ELBM_DIM 3
#define ELBM_SUFFIX d3q27
#define ELBM_PART 1
#include "elbm_kernels.cuh"
