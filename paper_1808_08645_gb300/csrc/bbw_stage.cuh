// bbw_stage.cuh -- fused BBWADG acoustic LSRK stage for sm_103a.
//
// One launch runs one stage of the five-stage low-storage RK4 (Sec. 6.3.1)
// over all elements. The paper splits a stage into volume, surface and update
// kernels (Sec. 6.3.1); here the three are one kernel, so each element's
// coefficients are read from HBM once per stage and its right-hand side never
// leaves shared memory.
//
// Work decomposition. Elements are processed in groups of V: the V elements
// of a group are interleaved in memory ([group][field][coefficient][V]) and
// every thread of the group's team of T lanes works on all V at once with
// vector loads and packed FP32x2 FMAs, so index arithmetic, table reads and
// barriers are paid once per V elements. A CTA holds GC teams that share the
// operator tables in shared memory and otherwise run independently: each
// team walks over groups with a grid-wide stride, staging one group at a time
// in its own shared region; the sparse Bernstein operators are gather stencils
// on the multi-index lattice driven by one packed word per output item
// (base index, lattice offsets, integer weights). Team phases are separated
// by __syncwarp (teams never span warps).
//
// Per group and stage:
//   V1/V2  grad p and div u (Sec. 4): degree N-1 combinations
//          w_beta = sum_m g_m a_{beta+e_m}, then one degree elevation
//          (E^N_{N-1}, Eq. 12) with integer weights gamma_j.
//   F      penalty fluxes of Eq. (2) on the 4 N_fp face coefficients, with the
//          neighbour traces gathered from q_in (L2),
//   L      then per face the lift L^f = E_L L0 (Sec. 4):
//          L0 = ((2N+3)/3) I + (N^2/3) E E^T on the face, and layer i of the
//          element receives ell_i (E^N_{N-i})^T L0 F,
//          ell_i = (-1)^i C(N,i)/(i+1), by i successive 2D reductions.
//   W      weight-adjusted update of the p right-hand side: Bernstein product
//          with c^2_M (Eq. 11 as a convolution of factorial-scaled
//          coefficients), M degree reductions, then P~_N of Eq. (20): a
//          downward reduction sweep whose levels stay in registers and an
//          upward elevation sweep scaled by c_j.
//   RK     res = a res + dt rhs, q_out = q_in + b res over the group with vector
//          loads and stores (stage 0 skips reading res, a_0 = 0); non-finite
//          values raise a status bit.
#pragma once

#include <cuda_runtime.h>

#include "bbw_common.h"

namespace bbw {

template <typename real>
struct StageParams {
  const real* __restrict__ qin;   // [G][4][Np][V]
  real* __restrict__ qout;        // [G][4][Np][V]
  real* __restrict__ res;         // [G][4][Np][V], updated in place
  const real* __restrict__ c2;    // [G][Mp][V]
  const real* __restrict__ geom;  // [G][9][V]: d lambda_m / d x_i, m = 1..3
  const int32_t* __restrict__ conn;  // [G][4][V] packed neighbour words
  const void* __restrict__ tables;   // Tables<N, M, real>
  int64_t G;                      // number of element groups
  real a, b, dt;
  real tau_p, tau_u;
  int64_t src_elem;               // -1: no source
  const real* __restrict__ src_vec;  // [Np]
  real src_amp;
  unsigned int* status;           // bit 0: non-finite output
};

template <typename real>
struct WadgParams {
  const real* __restrict__ rhs;  // [K][Np]
  const real* __restrict__ c2;   // [K][Mp]
  real* __restrict__ out;        // [K][Np]
  const void* __restrict__ tables;
  int64_t K;
};

// Launch shape per degree and precision: T lanes per group, V elements per
// group, GC groups per CTA.
template <int N, typename real>
struct TileShape;
template <int N>
struct TileShape<N, float> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : 32;
  static constexpr int V = N <= 5 ? 4 : 2;
  static constexpr int GC = N <= 2 ? 128 / T : N <= 4 ? 256 / T : N <= 6 ? 8 : 4;
};
template <int N>
struct TileShape<N, double> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : 32;
  static constexpr int V = N <= 4 ? 2 : 1;
  static constexpr int GC = N <= 4 ? 256 / T : N <= 6 ? 8 : 4;
};

// ---------------------------------------------------------------------------
// V-wide vectors of real. Float vectors of even width are stored as float2
// pairs so that arithmetic maps to the packed FP32x2 instructions of sm_100+.

template <typename real, int V>
struct vec {
  real x[V];
  __device__ __forceinline__ real get(int i) const { return x[i]; }
  __device__ __forceinline__ void set(int i, real v) { x[i] = v; }
};
template <int V>
struct vec2f {
  float2 h[V / 2];
  __device__ __forceinline__ float get(int i) const { return (i & 1) ? h[i >> 1].y : h[i >> 1].x; }
  __device__ __forceinline__ void set(int i, float v) {
    if (i & 1)
      h[i >> 1].y = v;
    else
      h[i >> 1].x = v;
  }
};
template <>
struct vec<float, 2> : vec2f<2> {};
template <>
struct vec<float, 4> : vec2f<4> {};

template <typename real, int V>
__device__ __forceinline__ vec<real, V> vzero() {
  vec<real, V> r;
#pragma unroll
  for (int i = 0; i < V; ++i) r.set(i, real(0));
  return r;
}

// shared/global vector load and store (V * sizeof(real) aligned)
template <typename real, int V>
__device__ __forceinline__ vec<real, V> vld(const real* p) {
  vec<real, V> r;
  if constexpr (V == 4 && sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.h[0] = make_float2(t.x, t.y);
    r.h[1] = make_float2(t.z, t.w);
  } else if constexpr (V == 2 && sizeof(real) == 4) {
    r.h[0] = *reinterpret_cast<const float2*>(p);
  } else if constexpr (V == 2 && sizeof(real) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r.x[0] = t.x;
    r.x[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) r.x[i] = p[i];
  }
  return r;
}
template <typename real, int V>
__device__ __forceinline__ void vst(real* p, const vec<real, V>& v) {
  if constexpr (V == 4 && sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v.h[0].x, v.h[0].y, v.h[1].x, v.h[1].y);
  } else if constexpr (V == 2 && sizeof(real) == 4) {
    *reinterpret_cast<float2*>(p) = v.h[0];
  } else if constexpr (V == 2 && sizeof(real) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v.x[0], v.x[1]);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) p[i] = v.x[i];
  }
}

// acc += a * b (elementwise)
template <typename real, int V>
__device__ __forceinline__ void vfma(vec<real, V>& acc, const vec<real, V>& a, const vec<real, V>& b) {
  if constexpr (sizeof(real) == 4 && V % 2 == 0) {
#pragma unroll
    for (int i = 0; i < V / 2; ++i) acc.h[i] = __ffma2_rn(a.h[i], b.h[i], acc.h[i]);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) acc.x[i] = fma(a.x[i], b.x[i], acc.x[i]);
  }
}
// acc += w * b (scalar w)
template <typename real, int V>
__device__ __forceinline__ void vfmas(vec<real, V>& acc, real w, const vec<real, V>& b) {
  if constexpr (sizeof(real) == 4 && V % 2 == 0) {
    const float2 ww = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < V / 2; ++i) acc.h[i] = __ffma2_rn(ww, b.h[i], acc.h[i]);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) acc.x[i] = fma(w, b.x[i], acc.x[i]);
  }
}
// w * a
template <typename real, int V>
__device__ __forceinline__ vec<real, V> vmuls(real w, const vec<real, V>& a) {
  vec<real, V> r;
  if constexpr (sizeof(real) == 4 && V % 2 == 0) {
    const float2 ww = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < V / 2; ++i) r.h[i] = __fmul2_rn(ww, a.h[i]);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) r.x[i] = w * a.x[i];
  }
  return r;
}
// a * b (elementwise)
template <typename real, int V>
__device__ __forceinline__ vec<real, V> vmul(const vec<real, V>& a, const vec<real, V>& b) {
  vec<real, V> r;
  if constexpr (sizeof(real) == 4 && V % 2 == 0) {
#pragma unroll
    for (int i = 0; i < V / 2; ++i) r.h[i] = __fmul2_rn(a.h[i], b.h[i]);
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) r.x[i] = a.x[i] * b.x[i];
  }
  return r;
}
// a + w * b
template <typename real, int V>
__device__ __forceinline__ vec<real, V> vaxpy(const vec<real, V>& a, real w, const vec<real, V>& b) {
  vec<real, V> r = a;
  vfmas(r, w, b);
  return r;
}
// a - b
template <typename real, int V>
__device__ __forceinline__ vec<real, V> vsub(const vec<real, V>& a, const vec<real, V>& b) {
  return vaxpy(a, real(-1), b);
}

// ---------------------------------------------------------------------------

template <int N, int M, typename real, int T, int V, int GC>
struct StageCfg {
  using Tab = Tables<N, M, real>;
  static constexpr int Np = np3(N);
  static constexpr int Nm1p = np3(N - 1);
  static constexpr int Nfp = np2(N);
  static constexpr int Mp = np3(M);
  static constexpr int NMp = np3(N + M);
  static constexpr int THREADS = T * GC;
  static constexpr int BUF = NMp > Np + 1 ? NMp : Np + 1;
  // scratch per group, in vectors: V1 (4 (N-1)_p), neighbour traces of the
  // four faces, later the fluxes and two lift pyramid levels (16 N_fp), WADG
  // ping-pong (2 BUF)
  static constexpr int S_VOL = 4 * Nm1p;
  static constexpr int S_LIFT = 16 * Nfp;
  static constexpr int S_WADG = 2 * BUF;
  static constexpr int S_SZ =
      S_VOL > S_LIFT ? (S_VOL > S_WADG ? S_VOL : S_WADG) : (S_LIFT > S_WADG ? S_LIFT : S_WADG);
  // per-team region, in vectors: Q [4][Np] | R [4][Np] | S | normals [4][4] |
  // c2 [Mp] | connectivity words [4][V] (int32); odd, so that teams start in
  // different shared-memory banks
  static constexpr int CONNV = (16 + int(sizeof(real)) - 1) / int(sizeof(real));
  static constexpr int TEAMV = (8 * Np + S_SZ + 16 + Mp + CONNV) | 1;
  static constexpr int TAB = table_bytes<N, M, real>();
  static constexpr int SMEM = TAB + int(sizeof(real)) * V * GC * TEAMV;
  static constexpr int RMAX = (Np + T - 1) / T;
  static constexpr int RK_IT = (4 * Np + T - 1) / T;  // RK vectors per lane
  static_assert(T >= 4 && T <= 32 && 32 % T == 0, "team must divide a warp and cover the 4 faces");
  static_assert(V == 1 || V == 2 || V == 4, "group width");
};

template <int T>
__device__ __forceinline__ void team_sync() {
  if constexpr (T > 1) __syncwarp();
}

struct Stencil3 {
  int base, dk, dl, w1, w2, w3;
};
__device__ __forceinline__ Stencil3 unpack_stencil3(uint32_t w) {
  return {int(w & 511u), int((w >> 9) & 15u), int((w >> 13) & 127u), int((w >> 20) & 15u),
          int((w >> 24) & 15u), int(w >> 28)};
}
struct Stencil2 {
  int base, db, w1, w2;
};
__device__ __forceinline__ Stencil2 unpack_stencil2(uint32_t w) {
  return {int(w & 127u), int((w >> 7) & 15u), int((w >> 11) & 15u), int((w >> 15) & 15u)};
}

// Copy the operator tables into shared memory (16-byte words).
template <int BYTES, int THREADS>
__device__ __forceinline__ void load_tables(unsigned char* dst, const void* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < BYTES / 16; i += THREADS) d[i] = s[i];
}

// Bulk prefetch of [p, p + bytes) into L2 (sm_90+); p 16-byte aligned.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  bytes &= ~15u;
  if (bytes && (reinterpret_cast<uintptr_t>(p) & 15u) == 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Asynchronous global -> shared copies (cp.async, sm_80+) of 4, 8 or 16 bytes.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const uint32_t s = uint32_t(__cvta_generic_to_shared(smem));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Weight-adjusted update of one group (Sec. 5): out = P^{N+M}_N (c2 * r).
// On entry A[0..Np) holds r * invfactN (A[Np] = 0) and bh the c2 coefficients
// scaled by invfactM. The result for items i = t + r*T is left in lv[0][r].
// A and B are vector buffers of BUF vectors each.
template <int N, int M, typename real, int T, int V, int RMAX>
__device__ __forceinline__ void wadg_group(const Tables<N, M, real>& tab, real* A, real* B,
                                           const vec<real, V> (&bh)[np3(M)], bool active, int t,
                                           vec<real, V> (&lv)[N + 1][RMAX]) {
  using vt = vec<real, V>;
  constexpr int Np = np3(N);
  constexpr int Mp = np3(M);
  constexpr int NMp = np3(N + M);
  // product h_gamma = gamma!/C(N+M,N) sum_beta (b_beta/beta!) (a_{gamma-beta}/(gamma-beta)!)
  for (int i = t; active && i < NMp; i += T) {
    const uint16_t* pr = tab.prod + i * Mp;
    vt h = vzero<real, V>();
#pragma unroll
    for (int b = 0; b < Mp; ++b) vfma(h, bh[b], vld<real, V>(A + pr[b] * V));
    vst(B + i * V, vmuls(tab.factNM[i], h));
  }
  team_sync<T>();
  // M one-degree reductions (E^{n}_{n-1})^T, n = N+M .. N+1 (right factors of Eq. 20)
  real* X = B;
  real* Y = A;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    const int n = N + M - r;
    const real inv = real(1) / real(n);
    for (int i = t; active && i < np3(n - 1); i += T) {
      const Stencil3 s = unpack_stencil3(tab.red3[off3(n - 1) + i]);
      vt v = vmuls(real(n + 3 - s.w1 - s.w2 - s.w3), vld<real, V>(X + s.base * V));
      vfmas(v, real(s.w1), vld<real, V>(X + (s.base + 1) * V));
      vfmas(v, real(s.w2), vld<real, V>(X + (s.base + s.dk) * V));
      vfmas(v, real(s.w3), vld<real, V>(X + (s.base + s.dl) * V));
      vst(Y + i * V, vmuls(inv, v));
    }
    real* tmp = X;
    X = Y;
    Y = tmp;
    team_sync<T>();
  }
  // v_0: the degree-N vector, kept per thread
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    const int i = t + r * T;
    lv[0][r] = (active && i < Np) ? vld<real, V>(X + i * V) : vzero<real, V>();
  }
  // downward sweep v_j = (E^{n}_{n-1})^T v_{j-1}, n = N-j+1
#pragma unroll
  for (int jl = 1; jl <= N; ++jl) {
    const int n = N - jl + 1;
    const real inv = real(1) / real(n);
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const int i = t + r * T;
      if (r * T < np3(n - 1) && active && i < np3(n - 1)) {
        const Stencil3 s = unpack_stencil3(tab.red3[off3(n - 1) + i]);
        vt v = vmuls(real(n + 3 - s.w1 - s.w2 - s.w3), vld<real, V>(X + s.base * V));
        vfmas(v, real(s.w1), vld<real, V>(X + (s.base + 1) * V));
        vfmas(v, real(s.w2), vld<real, V>(X + (s.base + s.dk) * V));
        vfmas(v, real(s.w3), vld<real, V>(X + (s.base + s.dl) * V));
        v = vmuls(inv, v);
        lv[jl][r] = v;
        vst(Y + i * V, v);
      }
    }
    real* tmp = X;
    X = Y;
    Y = tmp;
    team_sync<T>();
  }
  // upward sweep: w_N = c_N v_N, w_j = c_j v_j + E^{n}_{n-1} w_{j+1}, n = N-j
  if (active && t == 0) vst(X, vmuls(tab.cj[N], lv[N][0]));
  team_sync<T>();
#pragma unroll
  for (int jl = N - 1; jl >= 0; --jl) {
    const int n = N - jl;
    const real inv = real(1) / real(n);
    const real c = tab.cj[jl];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      const int i = t + r * T;
      if (r * T < np3(n) && active && i < np3(n)) {
        const Stencil3 s = unpack_stencil3(tab.elev3[off3(n) + i]);
        const int a0 = n - s.w1 - s.w2 - s.w3;
        vt acc = vzero<real, V>();
        if (a0 > 0) vfmas(acc, real(a0), vld<real, V>(X + s.base * V));
        if (s.w1 > 0) vfmas(acc, real(s.w1), vld<real, V>(X + (s.base - 1) * V));
        if (s.w2 > 0) vfmas(acc, real(s.w2), vld<real, V>(X + (s.base - s.dk) * V));
        if (s.w3 > 0) vfmas(acc, real(s.w3), vld<real, V>(X + (s.base - s.dl) * V));
        vt w = vmuls(c, lv[jl][r]);
        vfmas(w, inv, acc);
        if (jl > 0)
          vst(Y + i * V, w);
        else
          lv[0][r] = w;
      }
    }
    real* tmp = X;
    X = Y;
    Y = tmp;
    team_sync<T>();
  }
}

template <int N, int M, typename real, int T, int V, int GC>
__global__ void __launch_bounds__(T* GC) stage_kernel(const StageParams<real> P) {
  using C = StageCfg<N, M, real, T, V, GC>;
  using Tab = typename C::Tab;
  using vt = vec<real, V>;
  constexpr int Np = C::Np, Nm1p = C::Nm1p, Nfp = C::Nfp, Mp = C::Mp;
  constexpr int QV = 4 * Np;  // vectors of one state block of a group

  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  load_tables<C::TAB, C::THREADS>(smem, P.tables);
  __syncthreads();  // the only CTA-wide barrier: teams run independently below

  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  real* Q = reinterpret_cast<real*>(smem + C::TAB) + team * C::TEAMV * V;  // [4][Np]
  real* R = Q + QV * V;                                                   // [4][Np]
  real* S = R + QV * V;                                                   // scratch
  real* NRM = S + C::S_SZ * V;  // [4 faces][nx, ny, nz, (1/2)|f|/|D|]
  real* C2S = NRM + 16 * V;     // [Mp]
  int* CS = reinterpret_cast<int*>(C2S + Mp * V);  // [4][V]
  const int64_t G = P.G;
  const int64_t stride = int64_t(gridDim.x) * GC;
  const bool read_res = P.a != real(0);
  bool bad = false;

  for (int64_t g = int64_t(blockIdx.x) * GC + team; g < G; g += stride) {
    // the team's next group into L2
    if (t == 0 && g + stride < G) {
      const size_t qb = size_t(QV) * V * sizeof(real);
      prefetch_l2(P.qin + size_t(g + stride) * QV * V, uint32_t(qb));
      if (read_res) prefetch_l2(P.res + size_t(g + stride) * QV * V, uint32_t(qb));
    }
    // ---- stage the group: q, c2, connectivity into shared; geometry into registers ----
    {
      constexpr int VB = V * int(sizeof(real));  // bytes per vector: 4, 8 or 16
      const real* qg = P.qin + size_t(g) * QV * V;
      for (int idx = t; idx < QV; idx += T) cp_async<VB>(Q + idx * V, qg + size_t(idx) * V);
      for (int idx = t; idx < Mp; idx += T) cp_async<VB>(C2S + idx * V, P.c2 + (size_t(g) * Mp + idx) * V);
      for (int idx = t; idx < 4 * V; idx += T) cp_async<4>(CS + idx, P.conn + size_t(g) * 4 * V + idx);
    }
    vt gm[4][3];
#pragma unroll
    for (int m = 1; m < 4; ++m)
#pragma unroll
      for (int d = 0; d < 3; ++d) gm[m][d] = vld<real, V>(P.geom + (size_t(g) * 9 + 3 * (m - 1) + d) * V);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      gm[0][d] = vmuls(real(-1), gm[1][d]);
      gm[0][d] = vaxpy(gm[0][d], real(-1), gm[2][d]);
      gm[0][d] = vaxpy(gm[0][d], real(-1), gm[3][d]);
    }
    // face f = t: n = -g_f / |g_f|, (1/2) |f|/|D| = (3/2) |g_f|
    if (t < 4) {
      vt fx = gm[0][0], fy = gm[0][1], fz = gm[0][2];
#pragma unroll
      for (int m = 1; m < 4; ++m)
        if (t == m) {
          fx = gm[m][0];
          fy = gm[m][1];
          fz = gm[m][2];
        }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const real gx = fx.get(v), gy = fy.get(v), gz = fz.get(v);
        const real gn = sqrt(gx * gx + gy * gy + gz * gz);
        const real inv = real(1) / gn;
        real* nr = NRM + 4 * t * V + v;
        nr[0] = -gx * inv;
        nr[V] = -gy * inv;
        nr[2 * V] = -gz * inv;
        nr[3 * V] = real(1.5) * gn;
      }
    }
    cp_async_wait_all();
    team_sync<T>();

    // ---- V1: barycentric combinations at degree N-1, S = [4][Nm1p] ----
    for (int i = t; i < Nm1p; i += T) {
      const Stencil3 s = unpack_stencil3(tab.red3[off3(N - 1) + i]);
      const int im[4] = {s.base, s.base + 1, s.base + s.dk, s.base + s.dl};
      vt gx = vzero<real, V>(), gy = vzero<real, V>(), gz = vzero<real, V>(), dv = vzero<real, V>();
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const vt p = vld<real, V>(Q + im[m] * V);
        vfma(gx, gm[m][0], p);
        vfma(gy, gm[m][1], p);
        vfma(gz, gm[m][2], p);
        vfma(dv, gm[m][0], vld<real, V>(Q + (Np + im[m]) * V));
        vfma(dv, gm[m][1], vld<real, V>(Q + (2 * Np + im[m]) * V));
        vfma(dv, gm[m][2], vld<real, V>(Q + (3 * Np + im[m]) * V));
      }
      vst(S + i * V, gx);
      vst(S + (Nm1p + i) * V, gy);
      vst(S + (2 * Nm1p + i) * V, gz);
      vst(S + (3 * Nm1p + i) * V, dv);
    }
    team_sync<T>();
    // ---- V2: elevate to degree N; rhs_u = -grad p, rhs_p = -div u ----
    for (int i = t; i < Np; i += T) {
      const Stencil3 s = unpack_stencil3(tab.elev3[off3(N) + i]);
      const int a0 = N - s.w1 - s.w2 - s.w3;
      vt ax = vzero<real, V>(), ay = vzero<real, V>(), az = vzero<real, V>(), ad = vzero<real, V>();
      auto add = [&](int idx, int w) {
        const real wt = real(-w);
        vfmas(ax, wt, vld<real, V>(S + idx * V));
        vfmas(ay, wt, vld<real, V>(S + (Nm1p + idx) * V));
        vfmas(az, wt, vld<real, V>(S + (2 * Nm1p + idx) * V));
        vfmas(ad, wt, vld<real, V>(S + (3 * Nm1p + idx) * V));
      };
      if (a0 > 0) add(s.base, a0);
      if (s.w1 > 0) add(s.base - 1, s.w1);
      if (s.w2 > 0) add(s.base - s.dk, s.w2);
      if (s.w3 > 0) add(s.base - s.dl, s.w3);
      vst(R + i * V, ad);
      vst(R + (Np + i) * V, ax);
      vst(R + (2 * Np + i) * V, ay);
      vst(R + (3 * Np + i) * V, az);
    }
    team_sync<T>();

    // ---- F: neighbour traces of all four faces into NB = [field][4 Nfp]
    // (asynchronous 4-byte copies, many in flight), then the penalty fluxes
    // of Eq. (2) in place: F_p over field 0 and F_u over field 1 ----
    real* NB = S;
    for (int it = t; it < 4 * Nfp; it += T) {
      const int f = it / Nfp;
      const int a = it - f * Nfp;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = CS[f * V + v];
        if (c >= 0) {
          const int64_t nb = int64_t(c >> 5);
          const int ni = tab.nidx[(((c >> 3) & 3) * 6 + (c & 7)) * Nfp + a];
          const int64_t gq = nb / V;
          const real* src = P.qin + (size_t(gq) * QV + ni) * V + (nb - gq * V);
#pragma unroll
          for (int fld = 0; fld < 4; ++fld) cp_async<int(sizeof(real))>(NB + (fld * 4 * Nfp + it) * V + v, src + fld * Np * V);
        }
      }
    }
    cp_async_wait_all();
    for (int it = t; it < 4 * Nfp; it += T) {
      const int f = it / Nfp;
      const int io = tab.fidx[it];
      const vt pm = vld<real, V>(Q + io * V), um = vld<real, V>(Q + (Np + io) * V),
               vm = vld<real, V>(Q + (2 * Np + io) * V), wm = vld<real, V>(Q + (3 * Np + io) * V);
      vt pp = vld<real, V>(NB + it * V), up = vld<real, V>(NB + (4 * Nfp + it) * V),
         vp = vld<real, V>(NB + (8 * Nfp + it) * V), wp = vld<real, V>(NB + (12 * Nfp + it) * V);
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (CS[f * V + v] < 0) {  // p = 0 wall: mirror state
          pp.set(v, -pm.get(v));
          up.set(v, um.get(v));
          vp.set(v, vm.get(v));
          wp.set(v, wm.get(v));
        }
      const real* nr = NRM + 4 * f * V;
      const vt nx = vld<real, V>(nr), ny = vld<real, V>(nr + V), nz = vld<real, V>(nr + 2 * V),
               hs = vld<real, V>(nr + 3 * V);
      const vt jp = vsub(pp, pm);
      vt ndu = vmul(nx, vsub(up, um));
      vfma(ndu, ny, vsub(vp, vm));
      vfma(ndu, nz, vsub(wp, wm));
      vst(NB + it * V, vmul(hs, vaxpy(vmuls(P.tau_p, jp), real(-1), ndu)));
      vst(NB + (4 * Nfp + it) * V, vmul(hs, vaxpy(vmuls(P.tau_u, ndu), real(-1), jp)));
    }
    team_sync<T>();

    // ---- L: lift L^f = E_L L0 per face, accumulated into rhs ----
    {
      real* bufA = NB + 8 * Nfp * V;  // [p, u][Nfp], over the traces of fields 2, 3
      real* bufB = bufA + 2 * Nfp * V;
      const real third = real(1) / real(3);
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        const real* Fp = NB + f * Nfp * V;
        const real* Fu = NB + (4 * Nfp + f * Nfp) * V;
        const real* nr = NRM + 4 * f * V;
        const vt nx = vld<real, V>(nr), ny = vld<real, V>(nr + V), nz = vld<real, V>(nr + 2 * V);
        // t = E'^T F at degree N-1 (integer weights b_x + 1)
        for (int i = t; i < np2(N - 1); i += T) {
          const Stencil2 s = unpack_stencil2(tab.red2[off2(N - 1) + i]);
          const real w0 = real(N + 2 - s.w1 - s.w2), w1 = real(s.w1), w2 = real(s.w2);
          vt tp = vmuls(w0, vld<real, V>(Fp + s.base * V));
          vfmas(tp, w1, vld<real, V>(Fp + (s.base + 1) * V));
          vfmas(tp, w2, vld<real, V>(Fp + (s.base + s.db) * V));
          vt tu = vmuls(w0, vld<real, V>(Fu + s.base * V));
          vfmas(tu, w1, vld<real, V>(Fu + (s.base + 1) * V));
          vfmas(tu, w2, vld<real, V>(Fu + (s.base + s.db) * V));
          vst(bufB + i * V, tp);
          vst(bufB + (Nfp + i) * V, tu);
        }
        team_sync<T>();
        // g0 = L0 F = ((2N+3) F + E' t) / 3; layer 0 (ell_0 = 1)
        for (int i = t; i < Nfp; i += T) {
          const Stencil2 s = unpack_stencil2(tab.elev2[i]);
          const int a0 = N - s.w1 - s.w2;
          vt ep = vmuls(real(2 * N + 3), vld<real, V>(Fp + i * V));
          vt eu = vmuls(real(2 * N + 3), vld<real, V>(Fu + i * V));
          if (a0 > 0) {
            vfmas(ep, real(a0), vld<real, V>(bufB + s.base * V));
            vfmas(eu, real(a0), vld<real, V>(bufB + (Nfp + s.base) * V));
          }
          if (s.w1 > 0) {
            vfmas(ep, real(s.w1), vld<real, V>(bufB + (s.base - 1) * V));
            vfmas(eu, real(s.w1), vld<real, V>(bufB + (Nfp + s.base - 1) * V));
          }
          if (s.w2 > 0) {
            vfmas(ep, real(s.w2), vld<real, V>(bufB + (s.base - s.db) * V));
            vfmas(eu, real(s.w2), vld<real, V>(bufB + (Nfp + s.base - s.db) * V));
          }
          const vt gp = vmuls(third, ep);
          const vt gu = vmuls(third, eu);
          vst(bufA + i * V, gp);
          vst(bufA + (Nfp + i) * V, gu);
          real* r = R + tab.lidx[f * Np + i] * V;
          vst(r, vaxpy(vld<real, V>(r), real(1), gp));
          vt ru = vld<real, V>(r + Np * V);
          vfma(ru, nx, gu);
          vst(r + Np * V, ru);
          vt rv = vld<real, V>(r + 2 * Np * V);
          vfma(rv, ny, gu);
          vst(r + 2 * Np * V, rv);
          vt rw = vld<real, V>(r + 3 * Np * V);
          vfma(rw, nz, gu);
          vst(r + 3 * Np * V, rw);
        }
        team_sync<T>();
        real* cur = bufA;
        real* nxt = bufB;
        int off = Nfp;
#pragma unroll 1
        for (int layer = 1; layer <= N; ++layer) {
          const int n2 = N - layer;  // output degree; input degree n2 + 1
          const real scale = real(1) / real(n2 + 1);
          const real ell = tab.ell[layer] * scale;
          const vt enx = vmuls(ell, nx), eny = vmuls(ell, ny), enz = vmuls(ell, nz);
          for (int i = t; i < np2(n2); i += T) {
            const Stencil2 s = unpack_stencil2(tab.red2[off2(n2) + i]);
            const real w0 = real(n2 + 3 - s.w1 - s.w2), w1 = real(s.w1), w2 = real(s.w2);
            vt gp = vmuls(w0, vld<real, V>(cur + s.base * V));
            vfmas(gp, w1, vld<real, V>(cur + (s.base + 1) * V));
            vfmas(gp, w2, vld<real, V>(cur + (s.base + s.db) * V));
            vt gu = vmuls(w0, vld<real, V>(cur + (Nfp + s.base) * V));
            vfmas(gu, w1, vld<real, V>(cur + (Nfp + s.base + 1) * V));
            vfmas(gu, w2, vld<real, V>(cur + (Nfp + s.base + s.db) * V));
            // gp, gu are (n2+1) times the reduced values: the next level
            // stores them divided by n2+1, the scatter has 1/(n2+1) in ell
            vst(nxt + i * V, vmuls(scale, gp));
            vst(nxt + (Nfp + i) * V, vmuls(scale, gu));
            real* r = R + tab.lidx[f * Np + off + i] * V;
            vst(r, vaxpy(vld<real, V>(r), ell, gp));
            vt ru = vld<real, V>(r + Np * V);
            vfma(ru, enx, gu);
            vst(r + Np * V, ru);
            vt rv = vld<real, V>(r + 2 * Np * V);
            vfma(rv, eny, gu);
            vst(r + 2 * Np * V, rv);
            vt rw = vld<real, V>(r + 3 * Np * V);
            vfma(rw, enz, gu);
            vst(r + 3 * Np * V, rw);
          }
          off += np2(n2);
          real* tmp = cur;
          cur = nxt;
          nxt = tmp;
          team_sync<T>();
        }
      }
    }

    // ---- W: weight-adjusted update of the p right-hand side ----
    {
      real* A = S;
      real* B = S + C::BUF * V;
      const int src_lane = (P.src_elem >= 0 && P.src_elem / V == g) ? int(P.src_elem % V) : -1;
      for (int i = t; i < Np; i += T) {
        vt v = vld<real, V>(R + i * V);
        if (src_lane >= 0) {
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (l == src_lane) v.set(l, v.get(l) + P.src_amp * P.src_vec[i]);
        }
        vst(A + i * V, vmuls(tab.invfactN[i], v));
      }
      if (t == 0) vst(A + Np * V, vzero<real, V>());
      vt bh[Mp];
#pragma unroll
      for (int b = 0; b < Mp; ++b) bh[b] = vmuls(tab.invfactM[b], vld<real, V>(C2S + b * V));
      team_sync<T>();
      vt lv[N + 1][C::RMAX];
      wadg_group<N, M, real, T, V, C::RMAX>(tab, A, B, bh, true, t, lv);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (i < Np) vst(R + i * V, lv[0][r]);
      }
    }
    team_sync<T>();

    // ---- RK: res = a res + dt rhs; q_out = q_in + b res ([4][Np] vectors, coalesced) ----
    {
      real* resg = P.res + size_t(g) * QV * V;
      real* qog = P.qout + size_t(g) * QV * V;
      vt rold[C::RK_IT];  // all of this lane's res loads in flight at once
#pragma unroll
      for (int r = 0; r < C::RK_IT; ++r) {
        const int idx = t + r * T;
        rold[r] = (read_res && idx < QV) ? vld<real, V>(resg + size_t(idx) * V) : vzero<real, V>();
      }
#pragma unroll
      for (int r = 0; r < C::RK_IT; ++r) {
        const int idx = t + r * T;
        if (idx < QV) {
          vt rn = vmuls(P.dt, vld<real, V>(R + idx * V));
          vfmas(rn, P.a, rold[r]);
          vst(resg + size_t(idx) * V, rn);
          const vt qn = vaxpy(vld<real, V>(Q + idx * V), P.b, rn);
          vst(qog + size_t(idx) * V, qn);
#pragma unroll
          for (int v = 0; v < V; ++v) bad |= !isfinite(qn.get(v));
        }
      }
    }
    team_sync<T>();  // the next group reuses this team's shared region
  }
  if (bad) atomicOr(P.status, 1u);
}

// The weight-adjusted update alone: out = P^{N+M}_N (c2 * rhs) per element,
// on [K][Np] arrays (V consecutive elements form a group).
template <int N, int M, typename real, int T, int V, int GC>
__global__ void __launch_bounds__(T* GC) wadg_kernel(const WadgParams<real> P) {
  using C = StageCfg<N, M, real, T, V, GC>;
  using Tab = typename C::Tab;
  using vt = vec<real, V>;
  constexpr int Np = C::Np, Mp = C::Mp;
  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  load_tables<C::TAB, C::THREADS>(smem, P.tables);
  __syncthreads();
  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  real* R = reinterpret_cast<real*>(smem + C::TAB) + team * C::TEAMV * V;  // [Np]
  real* A = R + Np * V;
  real* B = A + C::BUF * V;
  real* C2S = B + C::BUF * V;  // [Mp]
  const int64_t G = (P.K + V - 1) / V;
  const int64_t stride = int64_t(gridDim.x) * GC;
  for (int64_t g = int64_t(blockIdx.x) * GC + team; g < G; g += stride) {
    const int64_t e0 = g * V;
    // gather [K][Np] into vectors; lanes past the last element get 0 and c2 = 1
    for (int idx = t; idx < V * Np; idx += T) {
      const int v = idx / Np, i = idx - v * Np;
      R[i * V + v] = e0 + v < P.K ? P.rhs[size_t(e0) * Np + idx] : real(0);
    }
    for (int idx = t; idx < V * Mp; idx += T) {
      const int v = idx / Mp, b = idx - v * Mp;
      C2S[b * V + v] = e0 + v < P.K ? P.c2[size_t(e0) * Mp + idx] : real(1);
    }
    team_sync<T>();
    for (int i = t; i < Np; i += T) vst(A + i * V, vmuls(tab.invfactN[i], vld<real, V>(R + i * V)));
    if (t == 0) vst(A + Np * V, vzero<real, V>());
    vt bh[Mp];
#pragma unroll
    for (int b = 0; b < Mp; ++b) bh[b] = vmuls(tab.invfactM[b], vld<real, V>(C2S + b * V));
    team_sync<T>();
    vt lv[N + 1][C::RMAX];
    wadg_group<N, M, real, T, V, C::RMAX>(tab, A, B, bh, true, t, lv);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int i = t + r * T;
      if (i < Np) vst(R + i * V, lv[0][r]);
    }
    team_sync<T>();
    for (int idx = t; idx < V * Np; idx += T) {
      const int v = idx / Np, i = idx - v * Np;
      if (e0 + v < P.K) P.out[size_t(e0) * Np + idx] = R[i * V + v];
    }
    team_sync<T>();
  }
}

}  // namespace bbw
