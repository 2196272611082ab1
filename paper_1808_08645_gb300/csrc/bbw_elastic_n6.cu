// Elastic stage kernels for degree N = 6.
#define BBW_N 6
#include "bbw_elastic_inst.cuh"
