// Elastic stage kernels for degree N = 9.
#define BBW_N 9
#include "bbw_elastic_inst.cuh"
