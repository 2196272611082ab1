// Elastic stage kernels for degree N = 3.
#define BBW_N 3
#include "bbw_elastic_inst.cuh"
