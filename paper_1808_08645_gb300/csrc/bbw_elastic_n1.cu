// Elastic stage kernels for degree N = 1.
#define BBW_N 1
#include "bbw_elastic_inst.cuh"
