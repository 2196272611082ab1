// Kernels of the BBWADG stage for degree N = 8.
#define BBW_N 8
#include "bbw_stage_inst.cuh"
