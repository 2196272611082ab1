// bbw_elastic_ops.h -- per-degree entry points of the elastic stage kernel,
// one table per N (1..kMaxN). Each bbw_elastic_n<N>.cu translation unit
// instantiates bbw_elastic.cuh for its N, every M in 0..kMaxM and both
// precisions. The operator tables are the acoustic ones (Tables<N, M, real>).
#pragma once

#include <cuda_runtime.h>

namespace bbw {

struct ElasticOps {
  // set the shared-memory attribute, return CTAs per SM of the stage kernel
  cudaError_t (*prepare)(int M, bool dbl, int* ctas_per_sm);
  // launch one stage; params points to ElasticParams<float|double>
  cudaError_t (*launch)(int M, bool dbl, const void* params, int grid, cudaStream_t s);
  // launch shape: lanes per group, elements per group, groups per CTA
  void (*shape)(int M, bool dbl, int* team, int* group_width, int* groups_per_cta);
};

const ElasticOps& elastic_ops_n1();
const ElasticOps& elastic_ops_n2();
const ElasticOps& elastic_ops_n3();
const ElasticOps& elastic_ops_n4();
const ElasticOps& elastic_ops_n5();
const ElasticOps& elastic_ops_n6();
const ElasticOps& elastic_ops_n7();
const ElasticOps& elastic_ops_n8();
const ElasticOps& elastic_ops_n9();

inline const ElasticOps* elastic_ops_for(int N) {
  switch (N) {
    case 1: return &elastic_ops_n1();
    case 2: return &elastic_ops_n2();
    case 3: return &elastic_ops_n3();
    case 4: return &elastic_ops_n4();
    case 5: return &elastic_ops_n5();
    case 6: return &elastic_ops_n6();
    case 7: return &elastic_ops_n7();
    case 8: return &elastic_ops_n8();
    case 9: return &elastic_ops_n9();
    default: return nullptr;
  }
}

}  // namespace bbw
