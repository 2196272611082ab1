// Elastic stage kernels for degree N = 8.
#define BBW_N 8
#include "bbw_elastic_inst.cuh"
