// Kernels of the BBWADG stage for degree N = 5.
#define BBW_N 5
#include "bbw_stage_inst.cuh"
