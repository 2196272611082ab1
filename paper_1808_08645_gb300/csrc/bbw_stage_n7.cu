// Kernels of the BBWADG stage for degree N = 7.
#define BBW_N 7
#include "bbw_stage_inst.cuh"
