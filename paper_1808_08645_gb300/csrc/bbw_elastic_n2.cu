// Elastic stage kernels for degree N = 2.
#define BBW_N 2
#include "bbw_elastic_inst.cuh"
