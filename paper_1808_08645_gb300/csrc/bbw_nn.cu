// bbw_nn.cu -- kernels of the neural-operator surrogate (the learned part
// that maps a c^2 field and a source position to receiver traces; the paper
// has no counterpart). Every dense contraction of the network, forward and
// backward, is one call of a batched GEMM on the BF16 tensor cores with FP32
// accumulation (mma.sync m16n8k16); the rest are elementwise, gather and
// optimiser kernels. Tensors are FP32 in memory; the GEMM rounds its operands
// to BF16 when it stages them into shared memory.
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

// C = alpha op(A) op(B) + beta C (+ bias[n]); op(A) is M x K, op(B) is K x N.
// A row-major M x K (lda) or, transposed, stored K x M; B row-major K x N
// (ldb) or, transposed, stored N x K. Batch b (blockIdx.z / splits) offsets
// A, B, C by sA, sB, sC elements. With splits > 1 the K range is divided
// among blockIdx.z % splits and the partial products are atomically added
// to C (beta and the bias must then be applied by the caller).
// Epilogue (splits == 1): pre (if set) receives the value before the
// activation; act = 1 applies GELU.
__global__ void __launch_bounds__(THREADS) gemm_bf16_kernel(const float* __restrict__ A, const float* __restrict__ B,
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
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // stage A tile [BM][BK] and B tile [BN][BK] as BF16
    for (int x = tid; x < BM * BK; x += THREADS) {
      const int mm = transA ? x % BM : x / BK, kk = transA ? x / BM : x % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[mm][kk] = __float2bfloat16_rn(v);
    }
    for (int x = tid; x < BN * BK; x += THREADS) {
      const int nn = transB ? x / BK : x % BN, kk = transB ? x % BK : x / BN;
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < kend) v = transB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bt[nn][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
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
    for (int h = 0; h < 4; ++h) {
      const int m = m0 + warp * 16 + g + (h >= 2 ? 8 : 0);
      const int n = n0 + j * 8 + tg * 2 + (h & 1);
      if (m >= M || n >= N) continue;
      float* c = C + (long long)m * ldc + n;
      float v = alpha * acc[j][h];
      if (splits > 1) {
        atomicAdd(c, v);
      } else {
        if (beta != 0.f) v += beta * *c;
        if (bias) v += bias[n];
        if (pre) pre[(long long)m * ldc + n] = v;
        *c = act == 1 ? gelu(v) : v;
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
  gemm_bf16_kernel<<<grid, THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
      A, B, C, bias, pre, M, N, K, lda, ldb, ldc, strideA, strideB, strideC, transA, transB, alpha, beta, act, splits);
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
