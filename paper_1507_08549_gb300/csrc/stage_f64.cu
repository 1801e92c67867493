// Double-precision instantiation of the stage kernels and helpers.
#define HYDRO_REAL double
#include "stage_inst.cuh"
