// Kernels of the BBWADG stage for degree N = 4.
#define BBW_N 4
#include "bbw_stage_inst.cuh"
