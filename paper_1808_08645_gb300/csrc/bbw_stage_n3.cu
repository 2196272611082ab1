// Kernels of the BBWADG stage for degree N = 3.
#define BBW_N 3
#include "bbw_stage_inst.cuh"
