// Kernels of the BBWADG stage for degree N = 1.
#define BBW_N 1
#include "bbw_stage_inst.cuh"
