// bbw_noalloc.cu -- bbw_wadg_update_noalloc: the weight-adjusted update with
// no device allocation.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being
// captured on another stream, frameworks that own the whole device pool and
// forbid allocations outside it, and real-time loops that must not block on the
// allocator. bbw_wadg_update gets its operator tables from a per-process cache
// that allocates device memory on first use of each (N, M, precision); this
// entry point instead keeps the tables of the current call in one fixed
// file-scope device array, so it never allocates or frees device memory. The
// tables reach that array through the parameters of an install kernel
// launched on the caller's stream ahead of the update kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "bbw_ops.h"
#include "bbw_stage.cuh"
#include "bbwadg.h"

namespace {

// Capacity of the static device scratch: the operator-table blob of one call.
// Every supported (N, M, precision) fits except N = 9 with M = 3 (34-37 KB).
constexpr size_t kScratchBytes = 32768;
constexpr int kMaxDevices = 64;

// Shared by every call in the process, on every device that loads the library
// (each device holds its own copy until the process exits). It keeps the
// tables of the last call; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_wadg_scratch[kScratchBytes];

// The tables travel to the device as the by-value parameter of a small
// install kernel (two launches of half the capacity each, under the kernel
// parameter limit), so nothing on the host is read after the launch returns.
constexpr size_t kChunkBytes = kScratchBytes / 2;
struct TableChunk {
  uint32_t offset, bytes;
  alignas(16) unsigned char data[kChunkBytes];
};

// chunk.bytes is a multiple of 16 (table blobs are) and offset + bytes <= kScratchBytes
__global__ void install_tables(const TableChunk chunk) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(chunk.data);
  uint32_t* dst = reinterpret_cast<uint32_t*>(g_wadg_scratch + chunk.offset);
  for (uint32_t i = threadIdx.x; i < chunk.bytes / 4; i += blockDim.x) dst[i] = src[i];
}

// Host staging for the tables (no heap allocation), guarded by g_mu.
alignas(16) unsigned char g_host_tables[kScratchBytes];
TableChunk g_chunk;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
// CTAs per SM of the WADG kernel per (device, N, M, precision), 0 = not prepared
int g_per_sm[kMaxDevices][bbw::kMaxN + 1][bbw::kMaxM + 1][2] = {};

bbw_status fail(bbw_status s, const char* what, cudaError_t err = cudaSuccess) {
  char msg[256];
  if (err != cudaSuccess)
    std::snprintf(msg, sizeof(msg), "bbw_wadg_update_noalloc: %s: %s", what, cudaGetErrorString(err));
  else
    std::snprintf(msg, sizeof(msg), "bbw_wadg_update_noalloc: %s", what);
  bbw::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" bbw_status bbw_wadg_update_noalloc(int N, int M, int precision, int64_t K, const void* rhs,
                                              const void* c2, void* out, void* stream) {
  if (N < 1 || N > bbw::kMaxN || M < 0 || M > bbw::kMaxM)
    return fail(BBW_ERR_UNSUPPORTED, "N must be in 1..9 and M in 0..3");
  if (precision != 32 && precision != 64) return fail(BBW_ERR_ARG, "precision must be 32 or 64");
  if (K < 0) return fail(BBW_ERR_ARG, "K < 0");
  if (K == 0) return BBW_OK;
  if (!rhs || !c2 || !out) return fail(BBW_ERR_ARG, "NULL device pointer");
  if (rhs == out) return fail(BBW_ERR_ARG, "out may not alias rhs");
  const bbw::KernelOps* ops = bbw::ops_for(N);
  const bool dbl = precision == 64;
  const size_t bytes = ops->table_bytes(M, dbl);
  if (bytes > kScratchBytes) {
    char what[160];
    std::snprintf(what, sizeof(what), "operator tables for N=%d, M=%d need %zu bytes, more than the %zu-byte static scratch",
                  N, M, bytes, kScratchBytes);
    return fail(BBW_ERR_ARG, what);
  }
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return fail(BBW_ERR_CUDA, "cudaGetDevice", err);
  if (dev < 0 || dev >= kMaxDevices) return fail(BBW_ERR_UNSUPPORTED, "device index beyond 63");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lock(g_mu);
  // once per device, with that device current: the device address of the scratch
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_wadg_scratch);
    if (err != cudaSuccess || !p) return fail(BBW_ERR_CUDA, "cudaGetSymbolAddress", err);
    int sms = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return fail(BBW_ERR_CUDA, "cudaDeviceGetAttribute", err);
    g_num_sms[dev] = std::max(1, sms);
    g_scratch_ptr[dev] = p;
  }
  int& per_sm = g_per_sm[dev][N][M][dbl ? 1 : 0];
  if (per_sm == 0) {
    int stage_per_sm = 0, wadg_per_sm = 0;
    err = ops->prepare(M, dbl, &stage_per_sm, &wadg_per_sm);
    if (err != cudaSuccess) return fail(BBW_ERR_CUDA, "kernel set-up", err);
    per_sm = std::max(1, wadg_per_sm);
  }
  // the tables of this call, copied over whatever the previous call left
  double cj[bbw::kMaxN + 1] = {};
  bbw_status st = bbw_projection_coeffs(N, M, cj);
  if (st != BBW_OK) return fail(st, "projection constants");
  std::memset(g_host_tables, 0, bytes);
  ops->build_tables(M, dbl, cj, g_host_tables);
  // the launch copies its parameter, so g_chunk may be refilled at once
  for (size_t off = 0; off < bytes; off += kChunkBytes) {
    g_chunk.offset = uint32_t(off);
    g_chunk.bytes = uint32_t(std::min(kChunkBytes, bytes - off));
    std::memcpy(g_chunk.data, g_host_tables + off, g_chunk.bytes);
    install_tables<<<1, 256, 0, s>>>(g_chunk);
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(BBW_ERR_CUDA, "table upload", err);
  }

  int team = 0, width = 1, gpc = 1;
  ops->launch_shape(M, dbl, &team, &width, &gpc);
  const int64_t per_cta = int64_t(width) * gpc;
  const int64_t tiles = (K + per_cta - 1) / per_cta;
  const int grid = int(std::min<int64_t>(tiles, int64_t(per_sm) * g_num_sms[dev]));
  if (dbl) {
    bbw::WadgParams<double> P{static_cast<const double*>(rhs), static_cast<const double*>(c2),
                              static_cast<double*>(out), g_scratch_ptr[dev], K};
    err = ops->launch_wadg(M, true, &P, grid, s);
  } else {
    bbw::WadgParams<float> P{static_cast<const float*>(rhs), static_cast<const float*>(c2),
                             static_cast<float*>(out), g_scratch_ptr[dev], K};
    err = ops->launch_wadg(M, false, &P, grid, s);
  }
  if (err != cudaSuccess) return fail(BBW_ERR_CUDA, "launch", err);
  return BBW_OK;
}
