// bbw_ops.h -- per-degree kernel entry points, one table per N (1..kMaxN).
// Each bbw_stage_n<N>.cu translation unit instantiates the templates of
// bbw_stage.cuh for its N, every M in 0..kMaxM and both precisions.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace bbw {

struct KernelOps {
  // bytes of the Tables<N, M, real> blob (16-byte multiple)
  size_t (*table_bytes)(int M, bool dbl);
  // fill a host buffer of table_bytes(M, dbl) bytes; cj has N+1 entries
  void (*build_tables)(int M, bool dbl, const double* cj, void* host_buf);
  // own face-node volume index fidx[4][Nfp] and neighbour index nidx[4 faces][6 codes][Nfp]
  void (*face_maps)(int* fidx, int* nidx);
  // set the shared-memory attribute, return CTAs per SM for the stage / wadg kernel
  cudaError_t (*prepare)(int M, bool dbl, int* stage_ctas_per_sm, int* wadg_ctas_per_sm);
  // launch one stage; params points to StageParams<float|double>
  cudaError_t (*launch_stage)(int M, bool dbl, const void* params, int grid, cudaStream_t s);
  // launch the weight-adjusted update; params points to WadgParams<float|double>
  cudaError_t (*launch_wadg)(int M, bool dbl, const void* params, int grid, cudaStream_t s);
  // launch shape: lanes per group, elements per group, groups per CTA
  void (*launch_shape)(int M, bool dbl, int* team, int* group_width, int* groups_per_cta);
  // launch the spatial operator alone (StageParams, output in qout)
  cudaError_t (*launch_spatial)(int M, bool dbl, const void* params, int grid, cudaStream_t s);
  // host-only: build the tables and check them against brute force (nullptr: all agree)
  const char* (*check_tables)(int M, bool dbl, const double* cj);
  // launch the adjoint stage's pre-kernel; params points to AdjPreParams<float|double>
  cudaError_t (*launch_adj_pre)(int M, bool dbl, const void* params, int grid, cudaStream_t s);
};

const KernelOps& ops_n1();
const KernelOps& ops_n2();
const KernelOps& ops_n3();
const KernelOps& ops_n4();
const KernelOps& ops_n5();
const KernelOps& ops_n6();
const KernelOps& ops_n7();
const KernelOps& ops_n8();
const KernelOps& ops_n9();

// Set the thread-local message returned by bbw_last_error() (defined in bbw_api.cu).
void set_last_error(const char* msg);

inline const KernelOps* ops_for(int N) {
  switch (N) {
    case 1: return &ops_n1();
    case 2: return &ops_n2();
    case 3: return &ops_n3();
    case 4: return &ops_n4();
    case 5: return &ops_n5();
    case 6: return &ops_n6();
    case 7: return &ops_n7();
    case 8: return &ops_n8();
    case 9: return &ops_n9();
    default: return nullptr;
  }
}

}  // namespace bbw
