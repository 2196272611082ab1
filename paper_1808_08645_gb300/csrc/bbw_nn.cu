// bbw_nn.cu -- kernels of the neural-operator surrogate (the learned part
// that maps a c^2 field and a source position to receiver traces; the paper
// has no counterpart). The dense contractions of the network, forward and
// backward, are calls of a batched GEMM on the BF16 tensor cores with FP32
// accumulation (mma.sync m16n8k16), except the transforms along the
// innermost spatial axis, which run as FP32 pencil kernels; the rest are
// elementwise, gather and optimiser kernels. Tensors are FP32 in memory; the
// GEMM rounds its operands to BF16 when it stages them into shared memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "bbw_ops.h"
#include "bbw_nn.h"

namespace {

bbw_status nn_fail(bbw_status s, const std::string& m) {
  bbw::set_last_error(("bbw_nn: " + m).c_str());
  return s;
}

#define NN_CUDA(call)                                                                           \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return nn_fail(BBW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int BM = 64, BN = 32, BK = 32;  // CTA tile; 4 warps of 16 x 32 each
constexpr int THREADS = 128;

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // low half = a
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Tile loaders: each thread holds its share of one op(A) tile (BM x BK, 16
// values) and one op(B) tile (BK x BN, 8 values) in registers, so that the
// next tile's global loads are in flight while the current one is multiplied.
// VEC: 16-byte loads along the operand's contiguous dimension (the caller
// guarantees a leading dimension, batch stride and base aligned to 4
// floats); ragged edges fall back to guarded scalar loads.
template <bool VEC>
__device__ __forceinline__ void load_a(float (&r)[16], const float* __restrict__ A, int lda, int transA, int M,
                                       int m0, int k0, int kend, int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * THREADS;  // 512 quads
      const int mm = transA ? (idx % 16) * 4 : idx / 8;
      const int kk = transA ? idx / 16 : (idx % 8) * 4;
      const int gm = m0 + mm, gk = k0 + kk;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!transA) {
        if (gm < M && gk + 3 < kend) {
          v = *reinterpret_cast<const float4*>(A + (long long)gm * lda + gk);
        } else if (gm < M) {
          const float* p = A + (long long)gm * lda;
          v.x = gk < kend ? p[gk] : 0.f;
          v.y = gk + 1 < kend ? p[gk + 1] : 0.f;
          v.z = gk + 2 < kend ? p[gk + 2] : 0.f;
          v.w = gk + 3 < kend ? p[gk + 3] : 0.f;
        }
      } else if (gk < kend) {
        const float* p = A + (long long)gk * lda;
        if (gm + 3 < M) {
          v = *reinterpret_cast<const float4*>(p + gm);
        } else {
          v.x = gm < M ? p[gm] : 0.f;
          v.y = gm + 1 < M ? p[gm + 1] : 0.f;
          v.z = gm + 2 < M ? p[gm + 2] : 0.f;
          v.w = gm + 3 < M ? p[gm + 3] : 0.f;
        }
      }
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = tid + q * THREADS;
      const int mm = transA ? x % BM : x / BK, kk = transA ? x / BM : x % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      r[q] = v;
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void store_a(const float (&r)[16], __nv_bfloat16 (*As)[BK + 8], int transA, int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * THREADS;
      const int mm = transA ? (idx % 16) * 4 : idx / 8;
      const int kk = transA ? idx / 16 : (idx % 8) * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (transA)
          As[mm + i][kk] = __float2bfloat16_rn(r[4 * q + i]);
        else
          As[mm][kk + i] = __float2bfloat16_rn(r[4 * q + i]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = tid + q * THREADS;
      const int mm = transA ? x % BM : x / BK, kk = transA ? x / BM : x % BK;
      As[mm][kk] = __float2bfloat16_rn(r[q]);
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void load_b(float (&r)[8], const float* __restrict__ B, int ldb, int transB, int N, int n0,
                                       int k0, int kend, int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int idx = tid + q * THREADS;  // 256 quads
      const int nn = transB ? idx / 8 : (idx % 8) * 4;
      const int kk = transB ? (idx % 8) * 4 : idx / 8;
      const int gn = n0 + nn, gk = k0 + kk;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (transB) {
        if (gn < N && gk + 3 < kend) {
          v = *reinterpret_cast<const float4*>(B + (long long)gn * ldb + gk);
        } else if (gn < N) {
          const float* p = B + (long long)gn * ldb;
          v.x = gk < kend ? p[gk] : 0.f;
          v.y = gk + 1 < kend ? p[gk + 1] : 0.f;
          v.z = gk + 2 < kend ? p[gk + 2] : 0.f;
          v.w = gk + 3 < kend ? p[gk + 3] : 0.f;
        }
      } else if (gk < kend) {
        const float* p = B + (long long)gk * ldb;
        if (gn + 3 < N) {
          v = *reinterpret_cast<const float4*>(p + gn);
        } else {
          v.x = gn < N ? p[gn] : 0.f;
          v.y = gn + 1 < N ? p[gn + 1] : 0.f;
          v.z = gn + 2 < N ? p[gn + 2] : 0.f;
          v.w = gn + 3 < N ? p[gn + 3] : 0.f;
        }
      }
      r[4 * q] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int x = tid + q * THREADS;
      const int nn = transB ? x / BK : x % BN, kk = transB ? x % BK : x / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < kend) v = transB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      r[q] = v;
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void store_b(const float (&r)[8], __nv_bfloat16 (*Bt)[BK + 8], int transB, int tid) {
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int idx = tid + q * THREADS;
      const int nn = transB ? idx / 8 : (idx % 8) * 4;
      const int kk = transB ? (idx % 8) * 4 : idx / 8;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (transB)
          Bt[nn][kk + i] = __float2bfloat16_rn(r[4 * q + i]);
        else
          Bt[nn + i][kk] = __float2bfloat16_rn(r[4 * q + i]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int x = tid + q * THREADS;
      const int nn = transB ? x / BK : x % BN, kk = transB ? x % BK : x / BN;
      Bt[nn][kk] = __float2bfloat16_rn(r[q]);
    }
  }
}

// C = alpha op(A) op(B) + beta C (+ bias[n]); op(A) is M x K, op(B) is K x N.
// A row-major M x K (lda) or, transposed, stored K x M; B row-major K x N
// (ldb) or, transposed, stored N x K. Batch b (blockIdx.z / splits) offsets
// A, B, C by sA, sB, sC elements. With splits > 1 the K range is divided
// among blockIdx.z % splits and the partial products are atomically added
// to C (beta and the bias must then be applied by the caller).
// Epilogue (splits == 1): pre (if set) receives the value before the
// activation; act = 1 applies GELU. VA / VB: 16-byte loads of A / B; VC:
// 8-byte stores of column pairs of C and pre (ldc, sC even, 8-byte bases).
template <bool VA, bool VB, bool VC>
__global__ void __launch_bounds__(THREADS, 4) gemm_bf16_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                           float* __restrict__ C, const float* __restrict__ bias,
                                                           float* __restrict__ pre, int M, int N, int K, int lda,
                                                           int ldb, int ldc, long long sA, long long sB,
                                                           long long sC, int transA, int transB, float alpha,
                                                           float beta, int act, int splits) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + 8];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bt[BN][BK + 8];  // [n][k]
  const int split = blockIdx.z % splits;
  const long long batch = blockIdx.z / splits;
  A += batch * sA;
  B += batch * sB;
  C += batch * sC;
  if (pre) pre += batch * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = lane >> 2, tg = lane & 3;
  float acc[4][4] = {};  // 4 n8 tiles x (c0..c3)
  float ra[16], rb[8];
  if (kbeg < kend) {
    load_a<VA>(ra, A, lda, transA, M, m0, kbeg, kend, tid);
    load_b<VB>(rb, B, ldb, transB, N, n0, kbeg, kend, tid);
  }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    store_a<VA>(ra, As, transA, tid);
    store_b<VB>(rb, Bt, transB, tid);
    __syncthreads();
    if (k0 + BK < kend) {  // the next tile's loads overlap this tile's products
      load_a<VA>(ra, A, lda, transA, M, m0, k0 + BK, kend, tid);
      load_b<VB>(rb, B, ldb, transB, N, n0, k0 + BK, kend, tid);
    }
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      const int r = warp * 16 + g;
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tg * 2]);
      a[1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tg * 2]);
      a[2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + tg * 2 + 8]);
      a[3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + tg * 2 + 8]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = j * 8 + g;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bt[n][ks + tg * 2]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bt[n][ks + tg * 2 + 8]);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int hp = 0; hp < 2; ++hp) {  // row g (hp = 0) or g + 8, columns n, n + 1
      const int m = m0 + warp * 16 + g + 8 * hp;
      const int n = n0 + j * 8 + tg * 2;
      if (m >= M || n >= N) continue;
      float v0 = alpha * acc[j][2 * hp], v1 = alpha * acc[j][2 * hp + 1];
      float* c = C + (long long)m * ldc + n;
      const bool two = n + 1 < N;
      if (splits > 1) {
        atomicAdd(c, v0);
        if (two) atomicAdd(c + 1, v1);
        continue;
      }
      if (VC && two) {
        if (beta != 0.f) {
          const float2 o = *reinterpret_cast<const float2*>(c);
          v0 += beta * o.x;
          v1 += beta * o.y;
        }
        if (bias) {
          v0 += bias[n];
          v1 += bias[n + 1];
        }
        if (pre) *reinterpret_cast<float2*>(pre + (long long)m * ldc + n) = make_float2(v0, v1);
        *reinterpret_cast<float2*>(c) = act == 1 ? make_float2(gelu(v0), gelu(v1)) : make_float2(v0, v1);
      } else {
        for (int h = 0; h < (two ? 2 : 1); ++h) {
          float v = h ? v1 : v0;
          if (beta != 0.f) v += beta * c[h];
          if (bias) v += bias[n + h];
          if (pre) pre[(long long)m * ldc + n + h] = v;
          c[h] = act == 1 ? gelu(v) : v;
        }
      }
    }
}

// Transform along one axis of pencils (the innermost spatial axis, channels
// contiguous): basis [L][m] in shared memory, FP32 on the CUDA cores. A
// thread takes one channel of PP consecutive pencils, so that every basis
// value it reads from shared memory serves PP products. expand = 0
// contracts, in [P][L][C] -> out [P][m][C], out[k] = sum_z basis[z][k] in[z];
// expand = 1 expands, in [P][m][C] -> out [P][L][C],
// v = sum_k basis[z][k] in[k] + beta out[z], pre[z] = v (if set),
// out[z] = act ? gelu(v) : v. Both read and write each value of the long
// side once: bound by HBM, not by arithmetic.
constexpr int kMaxModes = 16;
template <int MM, int PP>
__global__ void __launch_bounds__(256) axis_transform_kernel(const float* __restrict__ basis, int L, int m,
                                                            const float* __restrict__ in, float* __restrict__ out,
                                                            long long P, int C, int expand, float beta,
                                                            float* __restrict__ pre, int act) {
  extern __shared__ float phi[];  // [L][m]
  for (int x = threadIdx.x; x < L * m; x += blockDim.x) phi[x] = basis[x];
  __syncthreads();
  const long long PQ = (P + PP - 1) / PP;  // pencil quads
  const long long n = PQ * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long p0 = (i / C) * PP;
    const int c = int(i % C);
    const int np = P - p0 < PP ? int(P - p0) : PP;  // pencils of this thread (the last quad may be short)
    if (!expand) {
      float acc[PP][MM];
#pragma unroll
      for (int q = 0; q < PP; ++q)
#pragma unroll
        for (int k = 0; k < MM; ++k) acc[q][k] = 0.f;
      const float* src = in + p0 * L * C + c;
#pragma unroll 4
      for (int z = 0; z < L; ++z) {
        float u[PP];
#pragma unroll
        for (int q = 0; q < PP; ++q) u[q] = q < np ? src[((long long)q * L + z) * C] : 0.f;
#pragma unroll
        for (int k = 0; k < MM; ++k) {
          if (k < m) {
            const float w = phi[z * m + k];
#pragma unroll
            for (int q = 0; q < PP; ++q) acc[q][k] += w * u[q];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        if (q >= np) break;
        float* dst = out + ((p0 + q) * m) * C + c;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < m) dst[(long long)k * C] = acc[q][k];
      }
    } else {
      float t[PP][MM];
#pragma unroll
      for (int q = 0; q < PP; ++q)
#pragma unroll
        for (int k = 0; k < MM; ++k) t[q][k] = (q < np && k < m) ? in[((p0 + q) * m + k) * C + c] : 0.f;
      float* dst = out + p0 * L * C + c;
      float* pd = pre ? pre + p0 * L * C + c : nullptr;
      constexpr int ZC = 8;  // z values per chunk: all of a chunk's loads are issued before its stores
      for (int z0 = 0; z0 < L; z0 += ZC) {
        float o[ZC][PP];
#pragma unroll
        for (int zz = 0; zz < ZC; ++zz)
#pragma unroll
          for (int q = 0; q < PP; ++q)
            o[zz][q] = (beta != 0.f && q < np && z0 + zz < L) ? dst[((long long)q * L + z0 + zz) * C] : 0.f;
#pragma unroll
        for (int zz = 0; zz < ZC; ++zz) {
          const int z = z0 + zz;
          if (z >= L) break;
          float v[PP];
#pragma unroll
          for (int q = 0; q < PP; ++q) v[q] = beta != 0.f ? beta * o[zz][q] : 0.f;
#pragma unroll
          for (int k = 0; k < MM; ++k) {
            if (k < m) {
              const float w = phi[z * m + k];
#pragma unroll
              for (int q = 0; q < PP; ++q) v[q] += w * t[q][k];
            }
          }
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            if (q < np) {
              const long long off = ((long long)q * L + z) * C;
              if (pd) pd[off] = v[q];
              dst[off] = act == 1 ? gelu(v[q]) : v[q];
            }
          }
        }
      }
    }
  }
}

__global__ void gelu_backward_kernel(const float* __restrict__ pre, float* __restrict__ g, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    g[i] *= gelu_grad(pre[i]);
}

// db[n] += sum_m dY[m][n] (ldy = N): one thread per (column, row chunk);
// columns c0 + (threadIdx.x % W) for the block's column chunk c0 = blockIdx.y W
__global__ void bias_grad_kernel(const float* __restrict__ dY, float* __restrict__ db, long long Mrows, int N,
                                 int W) {
  const int n = blockIdx.y * W + threadIdx.x % W;
  const int lanes = blockDim.x / W;
  const int sub = threadIdx.x / W;
  if (n >= N) return;
  float acc = 0.f;
  for (long long m = (long long)blockIdx.x * lanes + sub; m < Mrows; m += (long long)gridDim.x * lanes)
    acc += dY[m * N + n];
  atomicAdd(db + n, acc);
}

// out[b][r][c] = (1/8) sum of the 2 x 2 x 2 grid points (rx[r] + {0,1},
// ry[r] + {0,1}, rz[r] + {0,1}) of u [B][X][Y][Z][C]; a stencil that does not
// lie inside the grid gives 0 (and is skipped by the transpose).
__device__ __forceinline__ bool stencil_ok(int x, int y, int z, int X, int Y, int Z) {
  return x >= 0 && y >= 0 && z >= 0 && x + 1 < X && y + 1 < Y && z + 1 < Z;
}

__global__ void gather_receivers_kernel(const float* __restrict__ u, float* __restrict__ out, const int* __restrict__ rx,
                                        const int* __restrict__ ry, const int* __restrict__ rz, int B, int X, int Y,
                                        int Z, int C, int R) {
  const long long n = (long long)B * R * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % C);
    const int r = int((i / C) % R);
    const long long b = i / ((long long)C * R);
    const int x0 = rx[r], y0 = ry[r], z0 = rz[r];
    float s = 0.f;
    if (stencil_ok(x0, y0, z0, X, Y, Z))
      for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
          for (int dz = 0; dz < 2; ++dz) s += u[((((b * X + x0 + dx) * Y) + y0 + dy) * Z + z0 + dz) * C + c];
    out[i] = 0.125f * s;
  }
}

// the transpose of gather_receivers (the receivers' stencils are disjoint)
__global__ void scatter_receivers_kernel(const float* __restrict__ gout, float* __restrict__ du,
                                         const int* __restrict__ rx, const int* __restrict__ ry,
                                         const int* __restrict__ rz, int B, int X, int Y, int Z, int C, int R) {
  const long long n = (long long)B * R * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % C);
    const int r = int((i / C) % R);
    const long long b = i / ((long long)C * R);
    const int x0 = rx[r], y0 = ry[r], z0 = rz[r];
    if (!stencil_ok(x0, y0, z0, X, Y, Z)) continue;
    for (int dx = 0; dx < 2; ++dx)
      for (int dy = 0; dy < 2; ++dy)
        for (int dz = 0; dz < 2; ++dz)
          du[((((b * X + x0 + dx) * Y) + y0 + dy) * Z + z0 + dz) * C + c] += 0.125f * gout[i];
  }
}

// out[i][t] = scale[i] * in[i] at the fractional sample t + shift[i]: linear
// interpolation between samples, the samples extended by zeros
__global__ void shift_traces_kernel(const float* __restrict__ in, float* __restrict__ out,
                                    const float* __restrict__ shift, const float* __restrict__ scale, long long rows,
                                    int T) {
  const long long n = rows * T;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / T;
    const int t = int(i % T);
    const float x = float(t) + shift[row];
    const float f = floorf(x);
    const float w = x - f;
    float v = 0.f;
    if (f >= 0.f && f <= float(T - 1)) {
      const int j = int(f);
      v = in[row * T + j] * (1.f - w);
      if (j + 1 < T) v += in[row * T + j + 1] * w;
    } else if (f == -1.f) {
      v = in[row * T] * w;
    }
    out[i] = (scale ? scale[row] : 1.f) * v;
  }
}

// loss += sum (y - t)^2 / n (one atomic per block), dy = 2 (y - t) / n
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                           float* __restrict__ loss, long long n) {
  __shared__ float part[32];
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    acc += d * d;
    if (dy) dy[i] = 2.f * d / float(n);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x % 32 == 0) part[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v / float(n));
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr_t m / (sqrt(v) + eps) with lr_t the bias-corrected step
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr_t, float b1, float b2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    p[i] -= lr_t * m[i] / (sqrtf(v[i]) + eps);
  }
}

int grid_for(long long n) { return int(std::min<long long>((n + 255) / 256, 152LL * 32)); }

}  // namespace

extern "C" {

bbw_status bbw_nn_gemm(int M, int N, int K, const float* A, int lda, long long strideA, int transA, const float* B,
                       int ldb, long long strideB, int transB, float* C, int ldc, long long strideC, int batch,
                       float alpha, float beta, const float* bias, float* pre, int act, int splits, void* stream) {
  if (M < 0 || N < 0 || K < 0 || batch < 1 || splits < 1 || splits > 1024)
    return nn_fail(BBW_ERR_ARG, "bad GEMM sizes");
  if (!A || !B || !C) return nn_fail(BBW_ERR_ARG, "NULL matrix");
  if (act != 0 && act != 1) return nn_fail(BBW_ERR_ARG, "act must be 0 (none) or 1 (GELU)");
  if (splits > 1 && (bias || pre || act || beta != 0.f))
    return nn_fail(BBW_ERR_ARG, "split-K accumulates into C: no bias, pre-activation, activation or beta");
  if ((long long)batch * splits > 65535) return nn_fail(BBW_ERR_ARG, "batch x splits beyond the grid limit");
  if (M == 0 || N == 0) return BBW_OK;
  const dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * splits);
  if (grid.y > 65535) return nn_fail(BBW_ERR_ARG, "M beyond the grid limit");
  // vector paths: the operand's rows (along its contiguous dimension) start on 16 bytes
  auto al = [](const void* p, unsigned a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
  const bool va = lda % 4 == 0 && strideA % 4 == 0 && al(A, 16);
  const bool vb = ldb % 4 == 0 && strideB % 4 == 0 && al(B, 16);
  const bool vc = ldc % 2 == 0 && strideC % 2 == 0 && al(C, 8) && (!pre || al(pre, 8));
  auto launch = [&](auto kern) {
    kern<<<grid, THREADS, 0, static_cast<cudaStream_t>(stream)>>>(A, B, C, bias, pre, M, N, K, lda, ldb, ldc, strideA,
                                                                   strideB, strideC, transA, transB, alpha, beta,
                                                                   act, splits);
  };
  if (va && vb)
    vc ? launch(gemm_bf16_kernel<true, true, true>) : launch(gemm_bf16_kernel<true, true, false>);
  else if (va)
    vc ? launch(gemm_bf16_kernel<true, false, true>) : launch(gemm_bf16_kernel<true, false, false>);
  else if (vb)
    vc ? launch(gemm_bf16_kernel<false, true, true>) : launch(gemm_bf16_kernel<false, true, false>);
  else
    vc ? launch(gemm_bf16_kernel<false, false, true>) : launch(gemm_bf16_kernel<false, false, false>);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_axis_transform(const float* basis, int L, int m, const float* in, float* out, long long pencils,
                                 int C, int expand, float beta, float* pre, int act, void* stream) {
  if (L < 1 || m < 1 || m > kMaxModes || C < 1 || pencils < 0 || (expand != 0 && expand != 1) ||
      (act != 0 && act != 1) || !basis || !in || !out || (!expand && (pre || act || beta != 0.f)))
    return nn_fail(BBW_ERR_ARG, "bad axis-transform arguments");
  if ((long long)L * m * sizeof(float) > 48 * 1024) return nn_fail(BBW_ERR_ARG, "axis-transform basis beyond 48 KB");
  if (pencils == 0) return BBW_OK;
  const size_t shm = size_t(L) * m * sizeof(float);
  auto launch = [&](auto kern, int pp) {
    const long long n = (pencils + pp - 1) / pp * C;
    const int blocks = int(std::min<long long>((n + 255) / 256, 152LL * 16));
    kern<<<blocks, 256, shm, static_cast<cudaStream_t>(stream)>>>(basis, L, m, in, out, pencils, C, expand, beta, pre,
                                                                   act);
  };
  if (m <= 8)
    launch(axis_transform_kernel<8, 4>, 4);
  else
    launch(axis_transform_kernel<16, 2>, 2);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_gelu_backward(const float* pre, float* grad, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!pre || !grad))) return nn_fail(BBW_ERR_ARG, "bad GELU arguments");
  if (n == 0) return BBW_OK;
  gelu_backward_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(pre, grad, n);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_bias_grad(const float* dY, float* db, long long rows, int N, void* stream) {
  if (rows < 0 || N < 1 || N > 65535 * 256 || !dY || !db) return nn_fail(BBW_ERR_ARG, "bad bias-gradient arguments");
  if (rows == 0) return BBW_OK;
  const int W = N <= 256 ? N : 256;  // columns per block
  const int lanes = 256 / W;
  const int blocks = int(std::min<long long>((rows + lanes - 1) / lanes, 152LL * 8));
  const dim3 grid(blocks, (N + W - 1) / W);
  bias_grad_kernel<<<grid, lanes * W, 0, static_cast<cudaStream_t>(stream)>>>(dY, db, rows, N, W);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_gather_receivers(const float* u, float* out, const int* rx, const int* ry, const int* rz, int B,
                                   int X, int Y, int Z, int C, int R, int transpose, void* stream) {
  if (B < 1 || X < 2 || Y < 2 || Z < 2 || C < 1 || R < 1 || !u || !out || !rx || !ry || !rz)
    return nn_fail(BBW_ERR_ARG, "bad receiver-gather arguments");
  const long long n = (long long)B * R * C;
  if (transpose)
    scatter_receivers_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        out, const_cast<float*>(u), rx, ry, rz, B, X, Y, Z, C, R);
  else
    gather_receivers_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(u, out, rx, ry, rz, B, X, Y,
                                                                                        Z, C, R);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_shift_traces(const float* in, float* out, const float* shift, const float* scale, long long rows,
                               int T, void* stream) {
  if (rows < 0 || T < 1 || (rows > 0 && (!in || !out || !shift)) || in == out)
    return nn_fail(BBW_ERR_ARG, "bad trace-shift arguments");
  if (rows == 0) return BBW_OK;
  const long long n = rows * T;
  shift_traces_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, shift, scale, rows, T);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_mse(const float* y, const float* t, float* dy, float* loss, long long n, void* stream) {
  if (n < 1 || !y || !t || !loss) return nn_fail(BBW_ERR_ARG, "bad MSE arguments");
  mse_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, t, dy, loss, n);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status bbw_nn_adam(float* p, const float* g, float* m, float* v, long long n, int step, float lr, float b1,
                       float b2, float eps, void* stream) {
  if (n < 0 || step < 1 || !(lr > 0.f) || (n > 0 && (!p || !g || !m || !v))) return nn_fail(BBW_ERR_ARG, "bad Adam arguments");
  if (n == 0) return BBW_OK;
  const float lr_t = lr * std::sqrt(1.f - std::pow(b2, float(step))) / (1.f - std::pow(b1, float(step)));
  adam_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(p, g, m, v, n, lr_t, b1, b2, eps);
  NN_CUDA(cudaGetLastError());
  return BBW_OK;
}

}  // extern "C"
