// Single-precision instantiation of the stage kernels and helpers.
#define HYDRO_REAL float
#define HYDRO_REAL_IS_FLOAT 1
#include "stage_inst.cuh"
