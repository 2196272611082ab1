// bbw_stage_inst.cuh -- instantiate the stage and WADG kernels for one degree.
// Included by bbw_stage_n<N>.cu with BBW_N defined.
#pragma once

#include <new>

#include "bbw_ops.h"
#include "bbw_stage.cuh"

#ifndef BBW_N
#error "define BBW_N before including bbw_stage_inst.cuh"
#endif

namespace bbw {
namespace {

constexpr int kN = BBW_N;

template <typename real>
using Shape = TileShape<kN, real>;

template <int M, typename real>
constexpr int kGC = fat_cta_groups<kN, M, real, Shape<real>::T, Shape<real>::V>();

template <int M, typename real>
using Cfg = StageCfg<kN, M, real, Shape<real>::T, Shape<real>::V, kGC<M, real>>;

template <int M, typename real>
constexpr auto stage_fn() {
  return stage_kernel<kN, M, real, Shape<real>::T, Shape<real>::V, kGC<M, real>>;
}
template <int M, typename real>
constexpr auto spatial_fn() {
  return stage_kernel<kN, M, real, Shape<real>::T, Shape<real>::V, kGC<M, real>, true>;
}
template <int M, typename real>
constexpr auto wadg_fn() {
  return wadg_kernel<kN, M, real, Shape<real>::T, Shape<real>::V, kGC<M, real>>;
}
template <int M, typename real>
constexpr auto adj_pre_fn() {
  return adj_pre_kernel<kN, M, real, Shape<real>::T, Shape<real>::V, kGC<M, real>>;
}


template <typename F>
auto dispatch(int M, bool dbl, F&& f) {
  switch (M) {
    case 0: return dbl ? f.template operator()<0, double>() : f.template operator()<0, float>();
    case 1: return dbl ? f.template operator()<1, double>() : f.template operator()<1, float>();
    case 2: return dbl ? f.template operator()<2, double>() : f.template operator()<2, float>();
    default: return dbl ? f.template operator()<3, double>() : f.template operator()<3, float>();
  }
}

void launch_shape(int M, bool dbl, int* team, int* width, int* groups) {
  dispatch(M, dbl, [&]<int MM, typename real>() {
    *team = Shape<real>::T;
    *width = Shape<real>::V;
    *groups = kGC<MM, real>;
    return 0;
  });
}

size_t tables_size(int M, bool dbl) {
  return dispatch(M, dbl, []<int MM, typename real>() { return size_t(Cfg<MM, real>::TAB); });
}

void build(int M, bool dbl, const double* cj, void* buf) {
  dispatch(M, dbl, [&]<int MM, typename real>() {
    auto* t = new (buf) Tables<kN, MM, real>();
    build_tables<kN, MM, real>(*t, cj);
    return 0;
  });
}

const char* check_tables(int M, bool dbl, const double* cj) {
  return dispatch(M, dbl, [&]<int MM, typename real>() -> const char* {
    auto* t = new Tables<kN, MM, real>();
    build_tables<kN, MM, real>(*t, cj);
    const char* msg = validate_tables<kN, MM, real>(*t);
    delete t;
    return msg;
  });
}

void face_maps(int* fidx, int* nidx) {
  auto* t = new Tables<kN, 0, double>();
  const double cj[kN + 1] = {};
  build_tables<kN, 0, double>(*t, cj);
  for (int i = 0; i < 4 * np2(kN); ++i) fidx[i] = t->fidx[i];
  for (int i = 0; i < 24 * np2(kN); ++i) nidx[i] = t->nidx[i];
  delete t;
}

cudaError_t prepare(int M, bool dbl, int* per_sm_stage, int* per_sm_wadg) {
  return dispatch(M, dbl, [&]<int MM, typename real>() {
    using C = Cfg<MM, real>;
    auto ks = stage_fn<MM, real>();
    auto kw = wadg_fn<MM, real>();
    cudaError_t err = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(spatial_fn<MM, real>(), cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(adj_pre_fn<MM, real>(), cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_stage, ks, C::THREADS, C::SMEM);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm_wadg, kw, C::THREADS, C::SMEM);
  });
}

cudaError_t launch_stage(int M, bool dbl, const void* params, int grid, cudaStream_t s) {
  return dispatch(M, dbl, [&]<int MM, typename real>() {
    using C = Cfg<MM, real>;
    stage_fn<MM, real>()<<<grid, C::THREADS, C::SMEM, s>>>(
        *static_cast<const StageParams<real>*>(params));
    return cudaGetLastError();
  });
}

cudaError_t launch_spatial(int M, bool dbl, const void* params, int grid, cudaStream_t s) {
  return dispatch(M, dbl, [&]<int MM, typename real>() {
    using C = Cfg<MM, real>;
    spatial_fn<MM, real>()<<<grid, C::THREADS, C::SMEM, s>>>(
        *static_cast<const StageParams<real>*>(params));
    return cudaGetLastError();
  });
}

cudaError_t launch_wadg(int M, bool dbl, const void* params, int grid, cudaStream_t s) {
  return dispatch(M, dbl, [&]<int MM, typename real>() {
    using C = Cfg<MM, real>;
    wadg_fn<MM, real>()<<<grid, C::THREADS, C::SMEM, s>>>(
        *static_cast<const WadgParams<real>*>(params));
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_pre(int M, bool dbl, const void* params, int grid, cudaStream_t s) {
  return dispatch(M, dbl, [&]<int MM, typename real>() {
    using C = Cfg<MM, real>;
    adj_pre_fn<MM, real>()<<<grid, C::THREADS, C::SMEM, s>>>(*static_cast<const AdjPreParams<real>*>(params));
    return cudaGetLastError();
  });
}

}  // namespace

#define BBW_CAT2(a, b) a##b
#define BBW_CAT(a, b) BBW_CAT2(a, b)
const KernelOps& BBW_CAT(ops_n, BBW_N)() {
  static const KernelOps ops = {&tables_size,  &build,          &face_maps,    &prepare,
                                &launch_stage, &launch_wadg,    &launch_shape, &launch_spatial,
                                &check_tables, &launch_adj_pre};
  return ops;
}

}  // namespace bbw
