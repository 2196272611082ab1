// Elastic stage kernels for degree N = 4.
#define BBW_N 4
#include "bbw_elastic_inst.cuh"
