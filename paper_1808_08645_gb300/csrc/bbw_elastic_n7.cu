// Elastic stage kernels for degree N = 7.
#define BBW_N 7
#include "bbw_elastic_inst.cuh"
