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
// by a team barrier: __syncwarp within a warp, a named barrier for teams of
// two warps.
//
// Per group and stage:
//   F1     neighbour traces of the four faces gathered from q_in (L2) with
//          asynchronous copies, in flight during V1;
//   V1     degree N-1 barycentric combinations for grad p and div u (Sec. 4):
//          w_beta = sum_m g_m a_{beta+e_m};
//   F2     penalty fluxes of Eq. (2) on the 4 N_fp face coefficients;
//   L      per face the lift pyramid of L^f = E_L L0 (Sec. 4):
//          L0 = ((2N+3)/3) I + (N^2/3) E E^T on the face, and level i,
//          ell_i (E^N_{N-i})^T L0 F with ell_i = (-1)^i C(N,i)/(i+1), by i
//          successive 2D reductions; every level of both fields is kept;
//   V2+L   per node: one degree elevation of V1 (E^N_{N-1}, Eq. 12, integer
//          weights) plus the node's four face contributions gathered from the
//          pyramids. The velocity fields finish their RK update here;
//   W      weight-adjusted update of the p right-hand side: Bernstein product
//          with c^2_M (Eq. 11 as a convolution of factorial-scaled
//          coefficients), M degree reductions, then P~_N of Eq. (20): a
//          downward reduction sweep whose levels stay in registers and an
//          upward elevation sweep scaled by c_j;
//   RK     res = a res + dt rhs, q_out = q_in + b res (stage 0 skips reading
//          res, a_0 = 0); non-finite values raise a status bit.
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
  // sources, listed by group: src_groups[j] (ascending) holds at least one
  // source element and src_slots[j][v] is the source of its element lane v
  // (-1: none); n_src_groups == 0: no sources. Source k adds
  // a_k src_vec[k][.] to the p right-hand side, with the host-given amplitude
  // sample a_k = src_amp[src_ser[k]][i] of sample i = 5 * step + stage
  // (0 for i >= n_amp), where step, the number of completed RK steps, is
  // *step_dev (device-resident, for replayed graphs) or step_host.
  int64_t n_src_groups;
  const int64_t* __restrict__ src_groups;  // [n_src_groups]
  const int32_t* __restrict__ src_slots;   // [n_src_groups][V]
  const real* __restrict__ src_vec;        // [nsrc][Np]
  const int32_t* __restrict__ src_ser;     // [nsrc] amplitude series of each source
  const double* __restrict__ src_amp;      // [nseries][n_amp]
  int64_t n_amp;
  const int64_t* step_dev;
  int64_t step_host;
  int stage;
  unsigned int* status;           // bit 0: non-finite output
  // LSRK stage: if set, the pressure bracket of the stage (volume term,
  // lifted fluxes and sources, before the weight-adjusted update) is also
  // stored here, [G][Np][V] (the adjoint's recomputed forward run keeps it).
  real* __restrict__ vout = nullptr;
  // spatial-only kernel: 0 writes the right-hand side to qout; 1 accumulates
  // qout -= dt |D| rhs into all four fields (|D| the element volume).
  int accumulate = 0;
  // per-group time steps (batches whose instances step with their own dt):
  // if set, group g uses dt_group[g] instead of dt; if steps_group is set, a
  // group whose step budget is used up (step >= steps_group[g], step as for
  // the sources) is left as it is: q_out = q_in, res untouched.
  const real* __restrict__ dt_group = nullptr;     // [G]
  const int64_t* __restrict__ steps_group = nullptr;  // [G]
};

// One stage of the discrete adjoint before its spatial operator, in the
// dual variables kap = M^{-1} qbar, rho = M^{-1} rbar of the state and
// residual cotangents (M the reference mass matrix, per element and field):
//   rho_t = a rho + b kap                       (stored back to rho)
//   y     = [P~(c2 rho_t,p) ; rho_t,u] / |D|    (the weight-adjusted update of Eq. 4)
template <typename real>
struct AdjPreParams {
  real* __restrict__ rho;         // [G][4][Np][V]
  const real* __restrict__ kap;   // [G][4][Np][V]
  const real* __restrict__ c2;    // [G][Mp][V]
  const real* __restrict__ geom;  // [G][9][V]
  real* __restrict__ y;           // [G][4][Np][V]
  const void* __restrict__ tables;
  int64_t G;
  real a, b;
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
// group. The number of groups per CTA is derived in StageCfg: as many teams
// as fit one CTA per SM (the operator tables are then held once per SM).
template <int N, typename real>
struct TileShape;
template <int N>
struct TileShape<N, float> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : N <= 7 ? 32 : 64;
  static constexpr int V = N <= 2 ? 2 : N <= 5 ? 4 : 2;  // measured: V = 2 is faster at N <= 2 only
};
template <int N>
struct TileShape<N, double> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : 32;
  static constexpr int V = N <= 4 ? 2 : 1;
};

constexpr int kSmemPerCta = 232448;  // 227 KB of dynamic shared memory per CTA (sm_100 family)

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
  // scratch per group, in vectors: the lift pyramids of p and u for the four
  // faces ([k][f][Np], level i at lift_level_base(N, i); level 0 first holds
  // the neighbour traces and fluxes), the degree N-1 combinations of V1
  // ([4][Nm1p]), and, when they do not fit beside level 0 in the pyramid
  // blocks (N < 3), the v and w neighbour traces ([2][4][Nfp]). The WADG
  // ping-pong buffers (2 BUF) reuse the region afterwards.
  static constexpr bool TR_IN_P = Np >= 2 * Nfp;
  static constexpr int S_PYR = 8 * Np;
  static constexpr int S_V1 = 4 * Nm1p;
  static constexpr int S_TR = TR_IN_P ? 0 : 8 * Nfp;
  static constexpr int S_LIFT = S_PYR + S_V1 + S_TR;
  static constexpr int S_SZ = S_LIFT > 2 * BUF ? S_LIFT : 2 * BUF;
  // per-team region, in vectors: Q [4][Np] | S | normals [4][4] | c2 [Mp] |
  // source amplitudes [V] | connectivity words [4][V] and source slots [V]
  // (int32, the slots written only for groups that hold a source); odd, so
  // that teams start in different shared-memory banks
  static constexpr int CONNV = 1 + (20 + int(sizeof(real)) - 1) / int(sizeof(real));
  static constexpr int TEAMV = (4 * Np + S_SZ + 16 + Mp + CONNV) | 1;
  static constexpr int TAB = table_bytes<N, M, real>();
  static constexpr int SMEM = TAB + int(sizeof(real)) * V * GC * TEAMV;
  static_assert(SMEM <= kSmemPerCta, "shared memory of the launch shape");
  static constexpr int RMAX = (Np + T - 1) / T;  // nodes per lane
  static_assert(T >= 4 && (T <= 32 ? 32 % T == 0 : T % 32 == 0), "team: a divisor or a multiple of a warp");
  static_assert(T <= 32 || GC <= 15, "one named barrier per multi-warp team");
  static_assert(V == 1 || V == 2 || V == 4, "group width");
};

// Barrier of one team: __syncwarp for teams within a warp, a named barrier
// (ids 1..15, one per team of the CTA) for teams of several warps.
// Teams per CTA. From N = 4 up: as many as fit the shared memory of one CTA
// per SM and 512 threads (so that 128 registers per thread fit the register
// file), which holds the operator tables once per SM. Below: 128-thread CTAs,
// several per SM (the tables are small there).
template <int N, int M, typename real, int T, int V>
constexpr int fat_cta_groups() {
  constexpr int team_bytes = int(sizeof(real)) * V * StageCfg<N, M, real, T, V, 1>::TEAMV;
  constexpr int by_smem = (kSmemPerCta - table_bytes<N, M, real>()) / team_bytes;
  constexpr int by_threads = (N <= 3 ? 128 : 512) / T;
  constexpr int g = by_smem < by_threads ? by_smem : by_threads;
  return T > 32 && g > 15 ? 15 : g;
}

template <int T>
__device__ __forceinline__ void team_sync() {
  if constexpr (T > 32) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + int(threadIdx.x) / T), "r"(T) : "memory");
  } else if constexpr (T > 1) {
    __syncwarp();
  }
}

// Checked build (BBW_CHECKED defined): indices that come from run-time data
// (the packed neighbour words) or from a table are range-checked before use;
// a failing check skips the access and raises status bit 1 (value 2). The
// normal build compiles none of it.
#ifdef BBW_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

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

// One-degree reduction (E^{n}_{n-1})^T into degree n-1 (outputs i = t + r*T)
// from X (degree n): every output of this lane is computed into out[] before
// anything is stored, so the lane's loads are all in flight together.
template <typename real, int V, int T, int R>
__device__ __forceinline__ void reduce_lane(const uint32_t* __restrict__ words, int count, int n,
                                            const real* X, int t, vec<real, V> (&out)[R]) {
  const real inv = real(1) / real(n);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = t + r * T;
    if (r * T < count && i < count) {
      const Stencil3 s = unpack_stencil3(words[i]);
      vec<real, V> v = vmuls(real(n + 3 - s.w1 - s.w2 - s.w3), vld<real, V>(X + s.base * V));
      vfmas(v, real(s.w1), vld<real, V>(X + (s.base + 1) * V));
      vfmas(v, real(s.w2), vld<real, V>(X + (s.base + s.dk) * V));
      vfmas(v, real(s.w3), vld<real, V>(X + (s.base + s.dl) * V));
      out[r] = vmuls(inv, v);
    }
  }
}

template <typename real, int V, int T, int R>
__device__ __forceinline__ void store_lane(real* Y, int count, int t, const vec<real, V> (&v)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = t + r * T;
    if (r * T < count && i < count) vst(Y + i * V, v[r]);
  }
}

// Weight-adjusted update of one group (Sec. 5): out = P^{N+M}_N (c2 * r).
// On entry A[0..Np) holds r * invfactN (A[Np] = 0) and bh the c2 coefficients
// scaled by invfactM. The result for items i = t + r*T is left in lv[0][r].
// A and B are vector buffers of BUF vectors each. Each phase computes all of
// a lane's outputs before storing them (loads in flight together).
template <int N, int M, typename real, int T, int V, int RMAX>
__device__ __forceinline__ void wadg_group(const Tables<N, M, real>& tab, real* A, real* B,
                                           const vec<real, V> (&bh)[np3(M)], bool active, int t,
                                           vec<real, V> (&lv)[N + 1][RMAX]) {
  using vt = vec<real, V>;
  constexpr int Np = np3(N);
  constexpr int Mp = np3(M);
  constexpr int NMp = np3(N + M);
  constexpr int RP = (NMp + T - 1) / T;  // outputs per lane of the product and reductions
  const int cnt = active ? 1 : 0;        // inactive teams produce nothing
  // product h_gamma = gamma!/C(N+M,N) sum_beta (b_beta/beta!) (a_{gamma-beta}/(gamma-beta)!)
  {
    vt h[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const int i = t + r * T;
      if (r * T < NMp && cnt && i < NMp) {
        vt acc = vzero<real, V>();
#pragma unroll
        for (int p = 0; p < (Mp + 1) / 2; ++p) {
          const uint32_t w = tab.prod2[p * NMp + i];
          vfma(acc, bh[2 * p], vld<real, V>(A + (w & 0xffffu) * V));
          if (2 * p + 1 < Mp) vfma(acc, bh[2 * p + 1], vld<real, V>(A + (w >> 16) * V));
        }
        h[r] = vmuls(tab.factNM[i], acc);
      }
    }
    store_lane<real, V, T, RP>(B, cnt * NMp, t, h);
  }
  team_sync<T>();
  // M one-degree reductions (E^{n}_{n-1})^T, n = N+M .. N+1 (right factors of Eq. 20)
  real* X = B;
  real* Y = A;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    const int n = N + M - r;
    vt out[RP];
    reduce_lane<real, V, T, RP>(tab.red3 + off3(n - 1), cnt * np3(n - 1), n, X, t, out);
    store_lane<real, V, T, RP>(Y, cnt * np3(n - 1), t, out);
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
    reduce_lane<real, V, T, RMAX>(tab.red3 + off3(n - 1), cnt * np3(n - 1), n, X, t, lv[jl]);
    store_lane<real, V, T, RMAX>(Y, cnt * np3(n - 1), t, lv[jl]);
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
    vt w[RMAX];
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
        w[r] = vmuls(c, lv[jl][r]);
        vfmas(w[r], inv, acc);
      }
    }
    if (jl > 0) {
      store_lane<real, V, T, RMAX>(Y, cnt * np3(n), t, w);
    } else {
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
        if (r * T < np3(n) && t + r * T < np3(n)) lv[0][r] = w[r];
    }
    real* tmp = X;
    X = Y;
    Y = tmp;
    team_sync<T>();
  }
}

// Amplitude sample of source sd at this stage (0 past the end of its series).
template <typename real>
__device__ __forceinline__ double stage_amplitude(const StageParams<real>& P, int sd) {
  const int64_t i = 5 * (P.step_dev ? *P.step_dev : P.step_host) + P.stage;
  return i < P.n_amp ? P.src_amp[size_t(P.src_ser[sd]) * size_t(P.n_amp) + size_t(i)] : 0.0;
}

// SP = false: one LSRK stage (above). SP = true: the spatial operator alone,
// for the adjoint: q_out receives [rhs_p before the weight-adjusted update
// (plus the point sources), rhs_u, rhs_v, rhs_w]; res, a, b and dt are not
// used.
template <int N, int M, typename real, int T, int V, int GC, bool SP = false>
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
  real* S = Q + QV * V;                                                   // scratch
  real* NRM = S + C::S_SZ * V;  // [4 faces][nx, ny, nz, (1/2)|f|/|D|]
  real* C2S = NRM + 16 * V;     // [Mp]
  real* AMP = C2S + Mp * V;                       // [V] source amplitude of this stage
  int* CS = reinterpret_cast<int*>(AMP + V);       // [4][V] connectivity, [V] source slots
  real* V1B = S + C::S_PYR * V;                    // [4][Nm1p]
  // slot of pyramid k (0: p, 1: u) of face f
  auto pyr = [&](int k, int f, int slot) { return S + ((k * 4 + f) * Np + slot) * V; };
  // neighbour trace of field fld at face node a of face f: p and u in level 0
  // of their pyramids (the fluxes replace them in place), v and w beside them
  auto trace = [&](int fld, int f, int a) -> real* {
    if (fld < 2) return pyr(fld, f, a);
    if constexpr (C::TR_IN_P)
      return pyr(fld - 2, f, Nfp + a);
    else
      return V1B + (C::S_V1 + ((fld - 2) * 4 + f) * Nfp + a) * V;
  };
  const int64_t G = P.G;
  const int64_t stride = int64_t(gridDim.x) * GC;
  const bool read_res = P.a != real(0);
  bool bad = false;
  bool oob = false;  // checked build only: an index out of range was met
  (void)oob;
  // cursor into the source groups: the first one at or after this team's
  // first group (the team's groups only increase; group indices fit 32 bits)
  const int nsg = int(P.n_src_groups);
  int js = 0;
  {
    int lo = 0, hi = nsg;
    const int64_t g0 = int64_t(blockIdx.x) * GC + team;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (P.src_groups[mid] < g0)
        lo = mid + 1;
      else
        hi = mid;
    }
    js = lo;
  }
  int next_src = js < nsg ? int(P.src_groups[js]) : INT32_MAX;
  const int64_t step_now = P.step_dev ? *P.step_dev : P.step_host;

  for (int64_t g = int64_t(blockIdx.x) * GC + team; g < G; g += stride) {
    if (P.steps_group && step_now >= P.steps_group[g]) {
      // the group's instance has taken its steps: carry its state over
      const real* qg = P.qin + size_t(g) * QV * V;
      real* og = P.qout + size_t(g) * QV * V;
      for (int idx = t; idx < QV; idx += T) vst(og + size_t(idx) * V, vld<real, V>(qg + size_t(idx) * V));
      continue;
    }
    const real dtg = P.dt_group ? P.dt_group[g] : P.dt;
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
    // the group's sources: slot (-1: none) and wavelet amplitude per element lane
    while (next_src < g) next_src = ++js < nsg ? int(P.src_groups[js]) : INT32_MAX;
    if (t < V) {
      const int sd = next_src == g ? P.src_slots[size_t(js) * V + t] : -1;
      CS[4 * V + t] = sd;
      if (sd >= 0) AMP[t] = real(stage_amplitude(P, sd));
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
    // accumulate mode of the spatial kernel: dt |D| per element lane, with
    // |D| = 1 / (6 det[grad lambda_1; grad lambda_2; grad lambda_3])
    vt dtvol = vzero<real, V>();
    if constexpr (SP) {
      if (P.accumulate) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const real a1 = gm[1][0].get(v), a2 = gm[1][1].get(v), a3 = gm[1][2].get(v);
          const real b1 = gm[2][0].get(v), b2 = gm[2][1].get(v), b3 = gm[2][2].get(v);
          const real c1 = gm[3][0].get(v), c2v = gm[3][1].get(v), c3 = gm[3][2].get(v);
          const real det = a1 * (b2 * c3 - b3 * c2v) - a2 * (b1 * c3 - b3 * c1) + a3 * (b1 * c2v - b2 * c1);
          dtvol.set(v, dtg / (real(6) * det));
        }
      }
    }
    cp_async_wait_all();
    team_sync<T>();

    // ---- F1: neighbour traces of all four faces (asynchronous 4- or 8-byte
    // copies from q_in in L2), in flight while V1 runs ----
    for (int it = t; it < 4 * Nfp; it += T) {
      const int f = it / Nfp;
      const int a = it - f * Nfp;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = CS[f * V + v];
        if (c >= 0) {
          const int64_t nb = int64_t(c >> 5);
          if constexpr (kChecked) {
            if (nb >= G * V || (c & 7) >= 6) {
              oob = true;
              continue;
            }
          }
          const int ni = tab.nidx[(((c >> 3) & 3) * 6 + (c & 7)) * Nfp + a];
          if constexpr (kChecked) {
            if (ni >= Np) {
              oob = true;
              continue;
            }
          }
          const int64_t gq = nb / V;
          const real* src = P.qin + (size_t(gq) * QV + ni) * V + (nb - gq * V);
#pragma unroll
          for (int fld = 0; fld < 4; ++fld) cp_async<int(sizeof(real))>(trace(fld, f, a) + v, src + fld * Np * V);
        }
      }
    }

    // ---- V1: barycentric combinations at degree N-1, V1B = [4][Nm1p] ----
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
      vst(V1B + i * V, gx);
      vst(V1B + (Nm1p + i) * V, gy);
      vst(V1B + (2 * Nm1p + i) * V, gz);
      vst(V1B + (3 * Nm1p + i) * V, dv);
    }
    cp_async_wait_all();
    team_sync<T>();

    // ---- F2: penalty fluxes of Eq. (2), in place over the p and u traces:
    // F_p into level 0 of the p pyramids, F_u into level 0 of the u pyramids ----
    {
      vt nf[4][4];  // per face: nx, ny, nz, (1/2)|f|/|D|
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int c = 0; c < 4; ++c) nf[f][c] = vld<real, V>(NRM + (4 * f + c) * V);
      for (int it = t; it < 4 * Nfp; it += T) {
        const int f = it / Nfp;
        const int a = it - f * Nfp;
        int io = tab.fidx[it];
        if constexpr (kChecked) {
          if (io >= Np) {
            oob = true;
            io = 0;
          }
        }
        const vt pm = vld<real, V>(Q + io * V), um = vld<real, V>(Q + (Np + io) * V),
                 vm = vld<real, V>(Q + (2 * Np + io) * V), wm = vld<real, V>(Q + (3 * Np + io) * V);
        vt pp = vld<real, V>(trace(0, f, a)), up = vld<real, V>(trace(1, f, a)),
           vp = vld<real, V>(trace(2, f, a)), wp = vld<real, V>(trace(3, f, a));
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (CS[f * V + v] < 0) {  // p = 0 wall: mirror state
            pp.set(v, -pm.get(v));
            up.set(v, um.get(v));
            vp.set(v, vm.get(v));
            wp.set(v, wm.get(v));
          }
        vt nx = nf[0][0], ny = nf[0][1], nz = nf[0][2], hs = nf[0][3];
#pragma unroll
        for (int ff = 1; ff < 4; ++ff)
          if (f == ff) {
            nx = nf[ff][0];
            ny = nf[ff][1];
            nz = nf[ff][2];
            hs = nf[ff][3];
          }
        const vt jp = vsub(pp, pm);
        vt ndu = vmul(nx, vsub(up, um));
        vfma(ndu, ny, vsub(vp, vm));
        vfma(ndu, nz, vsub(wp, wm));
        vst(trace(0, f, a), vmul(hs, vaxpy(vmuls(P.tau_p, jp), real(-1), ndu)));
        vst(trace(1, f, a), vmul(hs, vaxpy(vmuls(P.tau_u, ndu), real(-1), jp)));
      }
    }
    team_sync<T>();

    // ---- L: lift pyramids L^f = E_L L0 of the four faces (Sec. 4) ----
    // Level i of face f is ell_i (E^{N}_{N-i})^T L0 F_f; it lifts onto the
    // nodes with alpha_f = i. All levels of both fields are kept (stored
    // already scaled by ell_i), so that each node later gathers its four face
    // contributions once.
    {
      // t = E'^T F at degree N-1 (integer weights b_x + 1), beside level 0
      constexpr int CT = np2(N - 1);
      for (int it = t; it < 4 * CT; it += T) {
        const int f = it / CT;
        const int i = it - f * CT;
        const Stencil2 s = unpack_stencil2(tab.red2[off2(N - 1) + i]);
        const real w0 = real(N + 2 - s.w1 - s.w2), w1 = real(s.w1), w2 = real(s.w2);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          vt x = vmuls(w0, vld<real, V>(pyr(k, f, s.base)));
          vfmas(x, w1, vld<real, V>(pyr(k, f, s.base + 1)));
          vfmas(x, w2, vld<real, V>(pyr(k, f, s.base + s.db)));
          vst(pyr(k, f, Nfp + i), x);
        }
      }
      team_sync<T>();
      // level 0: L0 F = ((2N+3) F + E' t) / 3, in place over F
      const real third = real(1) / real(3);
      for (int it = t; it < 4 * Nfp; it += T) {
        const int f = it / Nfp;
        const int i = it - f * Nfp;
        const Stencil2 s = unpack_stencil2(tab.elev2[i]);
        const int a0 = N - s.w1 - s.w2;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          vt x = vmuls(real(2 * N + 3), vld<real, V>(pyr(k, f, i)));
          if (a0 > 0) vfmas(x, real(a0), vld<real, V>(pyr(k, f, Nfp + s.base)));
          if (s.w1 > 0) vfmas(x, real(s.w1), vld<real, V>(pyr(k, f, Nfp + s.base - 1)));
          if (s.w2 > 0) vfmas(x, real(s.w2), vld<real, V>(pyr(k, f, Nfp + s.base - s.db)));
          vst(pyr(k, f, i), vmuls(third, x));
        }
      }
      team_sync<T>();
      // levels 1..N: one 2D reduction each, times ell_i / ell_{i-1}
#pragma unroll 1
      for (int lv = 1; lv <= N; ++lv) {
        const int n2 = N - lv;  // output degree; input degree n2 + 1
        const int cnt = np2(n2);
        const int src = lift_level_base(N, lv - 1), dst = lift_level_base(N, lv);
        const real icnt = real(1) / real(cnt);
        const real scale = tab.lscale[lv];
        for (int it = t; it < 4 * cnt; it += T) {
          const int f = int((real(it) + real(0.5)) * icnt);
          const int i = it - f * cnt;
          const Stencil2 s = unpack_stencil2(tab.red2[off2(n2) + i]);
          const real w0 = real(n2 + 3 - s.w1 - s.w2) * scale, w1 = real(s.w1) * scale,
                     w2 = real(s.w2) * scale;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            vt x = vmuls(w0, vld<real, V>(pyr(k, f, src + s.base)));
            vfmas(x, w1, vld<real, V>(pyr(k, f, src + s.base + 1)));
            vfmas(x, w2, vld<real, V>(pyr(k, f, src + s.base + s.db)));
            vst(pyr(k, f, dst + i), x);
          }
        }
        team_sync<T>();
      }
    }

    // ---- V2 + lift gather per node: rhs_u = -grad p + sum_f n_f L^f F_u,
    // rhs_p = -div u + sum_f L^f F_p. The velocity fields finish their RK
    // update here (res = a res + dt rhs, q_out = q_in + b res); the p
    // right-hand side (plus the point source) goes on to the WADG update. ----
    real* resg = P.res + size_t(g) * QV * V;
    real* qog = P.qout + size_t(g) * QV * V;
    vt ap[C::RMAX];  // p right-hand side without the source
    {
      vt nrm[4][3];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int d = 0; d < 3; ++d) nrm[f][d] = vld<real, V>(NRM + (4 * f + d) * V);
      vt rold[C::RMAX][3];  // this lane's res loads, all in flight at once
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          rold[r][c] = (!SP && read_res && i < Np) ? vld<real, V>(resg + size_t((1 + c) * Np + i) * V)
                                                   : vzero<real, V>();
      }
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (i < Np) {
          const Stencil3 s = unpack_stencil3(tab.elev3[off3(N) + i]);
          const int a0 = N - s.w1 - s.w2 - s.w3;
          vt ad = vzero<real, V>(), rhs[3] = {vzero<real, V>(), vzero<real, V>(), vzero<real, V>()};
          auto add = [&](int idx, int w) {
            const real wt = real(-w);
            vfmas(rhs[0], wt, vld<real, V>(V1B + idx * V));
            vfmas(rhs[1], wt, vld<real, V>(V1B + (Nm1p + idx) * V));
            vfmas(rhs[2], wt, vld<real, V>(V1B + (2 * Nm1p + idx) * V));
            vfmas(ad, wt, vld<real, V>(V1B + (3 * Nm1p + idx) * V));
          };
          if (a0 > 0) add(s.base, a0);
          if (s.w1 > 0) add(s.base - 1, s.w1);
          if (s.w2 > 0) add(s.base - s.dk, s.w2);
          if (s.w3 > 0) add(s.base - s.dl, s.w3);
          const uint32_t lg = tab.lgat[i];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            int o = int((lg >> (8 * f)) & 255u);
            if constexpr (kChecked) {
              if (o >= Np) {
                oob = true;
                o = 0;
              }
            }
            const vt gu = vld<real, V>(pyr(1, f, o));
            ad = vaxpy(ad, real(1), vld<real, V>(pyr(0, f, o)));
#pragma unroll
            for (int d = 0; d < 3; ++d) vfma(rhs[d], nrm[f][d], gu);
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if constexpr (SP) {
              real* o = qog + size_t((1 + c) * Np + i) * V;
              if (P.accumulate) {
                vt acc = vld<real, V>(o);
                vfma(acc, vmuls(real(-1), dtvol), rhs[c]);
                vst(o, acc);
              } else {
                vst(o, rhs[c]);
              }
            } else {
              vt rn = vmuls(dtg, rhs[c]);
              vfmas(rn, P.a, rold[r][c]);
              vst(resg + size_t((1 + c) * Np + i) * V, rn);
              const vt qn = vaxpy(vld<real, V>(Q + ((1 + c) * Np + i) * V), P.b, rn);
              vst(qog + size_t((1 + c) * Np + i) * V, qn);
#pragma unroll
              for (int v = 0; v < V; ++v) bad |= !isfinite(qn.get(v));
            }
          }
          ap[r] = ad;
        }
      }
    }
    team_sync<T>();

    if constexpr (SP) {  // the p right-hand side before the weight-adjusted update
      bool any_src = false;
#pragma unroll
      for (int l = 0; l < V; ++l) any_src |= CS[4 * V + l] >= 0;
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (i < Np) {
          vt v = ap[r];
          if (any_src) {
#pragma unroll
            for (int l = 0; l < V; ++l) {
              const int sd = CS[4 * V + l];
              if (sd >= 0) v.set(l, v.get(l) + AMP[l] * P.src_vec[size_t(sd) * Np + i]);
            }
          }
          if (P.accumulate) {
            vt acc = vld<real, V>(qog + size_t(i) * V);
            vfma(acc, vmuls(real(-1), dtvol), v);
            vst(qog + size_t(i) * V, acc);
          } else {
            vst(qog + size_t(i) * V, v);
          }
        }
      }
    } else {
    // ---- W: weight-adjusted update of the p right-hand side, then its RK update ----
    {
      real* A = S;
      real* B = S + C::BUF * V;
      // plus the point sources, times 1 / alpha!
      bool any_src = false;
#pragma unroll
      for (int l = 0; l < V; ++l) any_src |= CS[4 * V + l] >= 0;
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (i < Np) {
          vt v = ap[r];
          if (any_src) {
#pragma unroll
            for (int l = 0; l < V; ++l) {
              const int sd = CS[4 * V + l];
              if (sd >= 0) v.set(l, v.get(l) + AMP[l] * P.src_vec[size_t(sd) * Np + i]);
            }
          }
          if (P.vout) vst(P.vout + (size_t(g) * Np + i) * V, v);
          vst(A + i * V, vmuls(tab.invfactN[i], v));
        }
      }
      if (t == 0) vst(A + Np * V, vzero<real, V>());
      vt bh[Mp];
#pragma unroll
      for (int b = 0; b < Mp; ++b) bh[b] = vmuls(tab.invfactM[b], vld<real, V>(C2S + b * V));
      team_sync<T>();
      vt lv[N + 1][C::RMAX];
      wadg_group<N, M, real, T, V, C::RMAX>(tab, A, B, bh, true, t, lv);
      vt rold[C::RMAX];
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        rold[r] = (read_res && i < Np) ? vld<real, V>(resg + size_t(i) * V) : vzero<real, V>();
      }
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (i < Np) {
          vt rn = vmuls(dtg, lv[0][r]);
          vfmas(rn, P.a, rold[r]);
          vst(resg + size_t(i) * V, rn);
          const vt qn = vaxpy(vld<real, V>(Q + i * V), P.b, rn);
          vst(qog + size_t(i) * V, qn);
#pragma unroll
          for (int v = 0; v < V; ++v) bad |= !isfinite(qn.get(v));
        }
      }
    }
    }
    team_sync<T>();  // the next group reuses this team's shared region
  }
  if (bad) atomicOr(P.status, 1u);
  if constexpr (kChecked) {
    if (oob) atomicOr(P.status, 2u);
  }
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

// The adjoint stage's update before its spatial operator (AdjPreParams).
template <int N, int M, typename real, int T, int V, int GC>
__global__ void __launch_bounds__(T* GC) adj_pre_kernel(const AdjPreParams<real> P) {
  using C = StageCfg<N, M, real, T, V, GC>;
  using Tab = typename C::Tab;
  using vt = vec<real, V>;
  constexpr int Np = C::Np, Mp = C::Mp;
  constexpr int BLK = 4 * Np * V;  // scalars of one group's four fields
  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  load_tables<C::TAB, C::THREADS>(smem, P.tables);
  __syncthreads();
  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  real* A = reinterpret_cast<real*>(smem + C::TAB) + team * C::TEAMV * V;
  real* B = A + C::BUF * V;
  real* C2S = B + C::BUF * V;  // [Mp]
  real* IV = C2S + Mp * V;     // [V] 1 / |D| per element lane
  const int64_t stride = int64_t(gridDim.x) * GC;
  for (int64_t g = int64_t(blockIdx.x) * GC + team; g < P.G; g += stride) {
    if (t < V) {  // 1 / |D| = 6 det[grad lambda_1; grad lambda_2; grad lambda_3]
      const real* gg = P.geom + size_t(g) * 9 * V + t;
      const real a1 = gg[0], a2 = gg[V], a3 = gg[2 * V], b1 = gg[3 * V], b2 = gg[4 * V], b3 = gg[5 * V],
                 c1 = gg[6 * V], c2v = gg[7 * V], c3 = gg[8 * V];
      IV[t] = real(6) * (a1 * (b2 * c3 - b3 * c2v) - a2 * (b1 * c3 - b3 * c1) + a3 * (b1 * c2v - b2 * c1));
    }
    for (int idx = t; idx < Mp * V; idx += T) C2S[idx] = P.c2[size_t(g) * Mp * V + idx];
    real* __restrict__ rg = P.rho + size_t(g) * BLK;
    const real* __restrict__ kg = P.kap + size_t(g) * BLK;
    real* __restrict__ yg = P.y + size_t(g) * BLK;
    // rho_t = a rho + b kap in vectors of V elements: all of a lane's NV
    // vector loads are issued before its stores
    constexpr int NV = (4 * Np + T - 1) / T;
    vt rv[NV];
#pragma unroll
    for (int r = 0; r < NV; ++r) {
      const int j = t + r * T;
      if (j < 4 * Np) rv[r] = vaxpy(vmuls(P.b, vld<real, V>(kg + size_t(j) * V)), P.a, vld<real, V>(rg + size_t(j) * V));
    }
    team_sync<T>();  // IV and C2S are ready
    const vt iv0 = vld<real, V>(IV);
#pragma unroll
    for (int r = 0; r < NV; ++r) {
      const int j = t + r * T;
      if (j < 4 * Np) {
        vst(rg + size_t(j) * V, rv[r]);
        if (j < Np)
          vst(A + j * V, vmuls(tab.invfactN[j], rv[r]));
        else
          vst(yg + size_t(j) * V, vmul(rv[r], iv0));
      }
    }
    if (t == 0) vst(A + Np * V, vzero<real, V>());
    vt bh[Mp];
#pragma unroll
    for (int b = 0; b < Mp; ++b) bh[b] = vmuls(tab.invfactM[b], vld<real, V>(C2S + b * V));
    team_sync<T>();
    vt lv[N + 1][C::RMAX];
    wadg_group<N, M, real, T, V, C::RMAX>(tab, A, B, bh, true, t, lv);
    const vt iv = vld<real, V>(IV);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int i = t + r * T;
      if (i < Np) vst(yg + size_t(i) * V, vmul(lv[0][r], iv));
    }
    team_sync<T>();
  }
}

}  // namespace bbw
