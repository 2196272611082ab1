// Kernels of the BBWADG stage for degree N = 9.
#define BBW_N 9
#include "bbw_stage_inst.cuh"
