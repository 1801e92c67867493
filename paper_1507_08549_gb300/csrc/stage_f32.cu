// Single-precision instantiation of the stage kernels and helpers.
#define HYDRO_REAL float
#include "stage_inst.cuh"
