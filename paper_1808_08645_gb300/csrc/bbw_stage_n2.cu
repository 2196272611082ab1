// Kernels of the BBWADG stage for degree N = 2.
#define BBW_N 2
#include "bbw_stage_inst.cuh"
