// bbw_elastic_inst.cuh -- instantiate the elastic stage kernel for one
// degree. Included by bbw_elastic_n<N>.cu with BBW_N defined.
#pragma once

#include "bbw_elastic.cuh"
#include "bbw_elastic_ops.h"

#ifndef BBW_N
#error "define BBW_N before including bbw_elastic_inst.cuh"
#endif

namespace bbw {
namespace {

constexpr int kN = BBW_N;

template <typename real>
using EShape = ElasticShape<kN, real>;

template <int M, typename real>
constexpr int kEGC = elastic_cta_groups<kN, M, real, EShape<real>::T, EShape<real>::V>();

template <int M, typename real>
using ECfg = ElasticCfg<kN, M, real, EShape<real>::T, EShape<real>::V, kEGC<M, real>>;

template <int M, typename real>
constexpr auto elastic_fn() {
  return elastic_stage_kernel<kN, M, real, EShape<real>::T, EShape<real>::V, kEGC<M, real>>;
}

template <typename F>
auto edispatch(int M, bool dbl, F&& f) {
  switch (M) {
    case 0: return dbl ? f.template operator()<0, double>() : f.template operator()<0, float>();
    case 1: return dbl ? f.template operator()<1, double>() : f.template operator()<1, float>();
    case 2: return dbl ? f.template operator()<2, double>() : f.template operator()<2, float>();
    default: return dbl ? f.template operator()<3, double>() : f.template operator()<3, float>();
  }
}

cudaError_t eprepare(int M, bool dbl, int* per_sm) {
  return edispatch(M, dbl, [&]<int MM, typename real>() {
    using C = ECfg<MM, real>;
    auto k = elastic_fn<MM, real>();
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, C::THREADS, C::SMEM);
  });
}

cudaError_t elaunch(int M, bool dbl, const void* params, int grid, cudaStream_t s) {
  return edispatch(M, dbl, [&]<int MM, typename real>() {
    using C = ECfg<MM, real>;
    elastic_fn<MM, real>()<<<grid, C::THREADS, C::SMEM, s>>>(*static_cast<const ElasticParams<real>*>(params));
    return cudaGetLastError();
  });
}

void eshape(int M, bool dbl, int* team, int* width, int* groups) {
  edispatch(M, dbl, [&]<int MM, typename real>() {
    *team = EShape<real>::T;
    *width = EShape<real>::V;
    *groups = kEGC<MM, real>;
    return 0;
  });
}

}  // namespace

#define BBW_ECAT2(a, b) a##b
#define BBW_ECAT(a, b) BBW_ECAT2(a, b)
const ElasticOps& BBW_ECAT(elastic_ops_n, BBW_N)() {
  static const ElasticOps ops = {&eprepare, &elaunch, &eshape};
  return ops;
}

}  // namespace bbw
