// Kernels of the BBWADG stage for degree N = 6.
#define BBW_N 6
#include "bbw_stage_inst.cuh"
