// Double-precision instantiation of the stage kernels and helpers.
#define HYDRO_REAL double
#define HYDRO_REAL_IS_FLOAT 0
#include "stage_inst.cuh"
