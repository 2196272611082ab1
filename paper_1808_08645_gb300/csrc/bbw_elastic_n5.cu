// Elastic stage kernels for degree N = 5.
#define BBW_N 5
#include "bbw_elastic_inst.cuh"
