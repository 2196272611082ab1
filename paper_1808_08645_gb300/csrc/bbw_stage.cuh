// bbw_stage.cuh -- fused BBWADG acoustic LSRK stage for sm_103a.
//
// One launch runs one stage of the five-stage low-storage RK4 (Sec. 6.3.1)
// over all elements. The paper splits a stage into volume, surface and update
// kernels (Sec. 6.3.1); here the three are one kernel so that each element's
// coefficients are read from HBM once and its right-hand side never leaves
// shared memory.
//
// Work decomposition: a persistent CTA walks over tiles of E consecutive
// elements; a team of T threads owns one element of the tile. Tile data is
// staged in shared memory with an odd per-element stride; the sparse Bernstein
// operators are applied as gather stencils on the multi-index lattice, each
// thread producing output coefficients i = t, t+T, t+2T, ... of a phase, with
// neighbour indices computed from the decoded multi-index (closed-form index
// arithmetic, no CSR loads). Phases of one element are separated by team
// barriers (__syncwarp for T <= 32).
//
// Per element and stage:
//   V1/V2  grad p and div u (Sec. 4): degree N-1 barycentric combinations
//          w_beta = sum_m g_m a_{beta+e_m}, then one degree elevation
//          (E^N_{N-1}, Eq. 12) with integer weights gamma_j.
//   F      penalty fluxes of Eq. (2) on the 4 x N_fp face coefficients;
//          neighbour traces come from shared memory when the neighbour is in
//          the tile, else from q_in in global memory.
//   L      lift L^f = E_L L0 (Sec. 4): L0 = ((2N+3)/3) I + (N^2/3) E E^T on
//          the face, then layer i of the element receives
//          ell_i (E^N_{N-i})^T L0 F with ell_i = (-1)^i C(N,i)/(i+1),
//          evaluated as i successive 2D one-degree reductions.
//   W      weight-adjusted update of the p right-hand side: Bernstein product
//          with c^2_M (Eq. 11, as a convolution of factorial-scaled
//          coefficients), M degree reductions, then P~_N of Eq. (20) by a
//          downward reduction sweep (levels kept in registers) and an upward
//          elevation sweep scaled by c_j.
//   RK     res = a res + dt rhs, q_out = q_in + b res (stage 0 skips reading
//          res because a_0 = 0), coalesced over the tile; non-finite values
//          raise a status bit.
#pragma once

#include <cuda_runtime.h>

#include "bbw_common.h"

namespace bbw {

template <typename real>
struct StageParams {
  const real* __restrict__ qin;   // [4][K][Np]
  real* __restrict__ qout;        // [4][K][Np]
  real* __restrict__ res;         // [4][K][Np], updated in place
  const real* __restrict__ c2;    // [K][Mp]
  const real* __restrict__ geom;  // [K][9]: d lambda_m / d x_i, m = 1..3
  const int32_t* __restrict__ conn;  // [K][4] packed neighbour words
  const void* __restrict__ tables;   // Tables<N, M, real>
  int64_t K;
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

// Launch shape per degree: T threads per element, E elements per CTA.
template <int N>
struct TileShape {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : 32;
  static constexpr int E = 256 / T;
};

template <int N, int M, typename real, int T, int E>
struct StageCfg {
  using Tab = Tables<N, M, real>;
  static constexpr int Np = np3(N);
  static constexpr int Nm1p = np3(N - 1);
  static constexpr int Nfp = np2(N);
  static constexpr int Mp = np3(M);
  static constexpr int NMp = np3(N + M);
  static constexpr int THREADS = T * E;
  static constexpr int BUF = NMp > Np + 1 ? NMp : Np + 1;
  static constexpr int S_VOL = 4 * Nm1p;
  static constexpr int S_LIFT = 12 * Nfp;
  static constexpr int S_WADG = 2 * BUF;
  static constexpr int S_SZ =
      S_VOL > S_LIFT ? (S_VOL > S_WADG ? S_VOL : S_WADG) : (S_LIFT > S_WADG ? S_LIFT : S_WADG);
  static constexpr int STRIDE = (8 * Np + S_SZ) | 1;  // odd: spreads elements over banks
  static constexpr int GEO = 28;  // g[4][3] then (nx, ny, nz, |f|/|D|) per face
  static constexpr int TAB = table_bytes<N, M, real>();
  static constexpr int SMEM =
      TAB + int(sizeof(real)) * (E * STRIDE + E * GEO + E * Mp) + 4 * E * 4;
  static constexpr int RMAX = (Np + T - 1) / T;
  static_assert(T <= 32 && 32 % T == 0, "team must divide a warp");
};

template <int T>
__device__ __forceinline__ void team_sync() {
  if constexpr (T > 1) __syncwarp();
}

__device__ __forceinline__ void unpack4(uint32_t w, int& a0, int& a1, int& a2, int& a3) {
  a0 = int(w & 255u);
  a1 = int((w >> 8) & 255u);
  a2 = int((w >> 16) & 255u);
  a3 = int(w >> 24);
}

// Copy the operator tables into shared memory (16-byte words).
template <int BYTES, int THREADS>
__device__ __forceinline__ void load_tables(unsigned char* dst, const void* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < BYTES / 16; i += THREADS) d[i] = s[i];
}

// Weight-adjusted update of one element (Sec. 5): out = P^{N+M}_N (c2 * r).
// On entry A[0..Np) holds r * invfactN (A[Np] = 0), bh the c2 coefficients
// scaled by invfactM. The result for items i = t + r*T is left in lv[0][r].
template <int N, int M, typename real, int T, int RMAX>
__device__ __forceinline__ void wadg_element(const Tables<N, M, real>& tab, real* A, real* B,
                                             const real (&bh)[np3(M) > 0 ? np3(M) : 1],
                                             bool active, int t, real (&lv)[N + 1][RMAX]) {
  constexpr int Np = np3(N);
  constexpr int Mp = np3(M);
  constexpr int NMp = np3(N + M);
  // product h_gamma = gamma!/C(N+M,N) sum_beta (b_beta/beta!) (a_{gamma-beta}/(gamma-beta)!)
  for (int i = t; active && i < NMp; i += T) {
    const uint16_t* pr = tab.prod + i * Mp;
    real h = real(0);
#pragma unroll
    for (int b = 0; b < Mp; ++b) h += bh[b] * A[pr[b]];
    B[i] = h * tab.factNM[i];
  }
  team_sync<T>();
  // M one-degree reductions (E^{n}_{n-1})^T, n = N+M .. N+1 (Eq. 20, right factors)
  real* X = B;
  real* Y = A;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    const int n = N + M - r;
    const real inv = real(1) / real(n);
    for (int i = t; active && i < np3(n - 1); i += T) {
      int b0, j, k, l;
      unpack4(tab.dec3[off3(n - 1) + i], b0, j, k, l);
      const real v = real(b0 + 1) * X[idx3(n, j, k, l)] + real(j + 1) * X[idx3(n, j + 1, k, l)] +
                     real(k + 1) * X[idx3(n, j, k + 1, l)] + real(l + 1) * X[idx3(n, j, k, l + 1)];
      Y[i] = v * inv;
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
    lv[0][r] = (active && i < Np) ? X[i] : real(0);
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
        int b0, j, k, l;
        unpack4(tab.dec3[off3(n - 1) + i], b0, j, k, l);
        const real v = (real(b0 + 1) * X[idx3(n, j, k, l)] + real(j + 1) * X[idx3(n, j + 1, k, l)] +
                        real(k + 1) * X[idx3(n, j, k + 1, l)] +
                        real(l + 1) * X[idx3(n, j, k, l + 1)]) *
                       inv;
        lv[jl][r] = v;
        Y[i] = v;
      }
    }
    real* tmp = X;
    X = Y;
    Y = tmp;
    team_sync<T>();
  }
  // upward sweep: w_N = c_N v_N, w_j = c_j v_j + E^{n}_{n-1} w_{j+1}, n = N-j
  if (active && t == 0) X[0] = tab.cj[N] * lv[N][0];
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
        int a0, j, k, l;
        unpack4(tab.dec3[off3(n) + i], a0, j, k, l);
        real acc = real(0);
        if (a0 > 0) acc += real(a0) * X[idx3(n - 1, j, k, l)];
        if (j > 0) acc += real(j) * X[idx3(n - 1, j - 1, k, l)];
        if (k > 0) acc += real(k) * X[idx3(n - 1, j, k - 1, l)];
        if (l > 0) acc += real(l) * X[idx3(n - 1, j, k, l - 1)];
        const real w = c * lv[jl][r] + acc * inv;
        if (jl > 0)
          Y[i] = w;
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

template <int N, int M, typename real, int T, int E>
__global__ void __launch_bounds__(T* E) stage_kernel(const StageParams<real> P) {
  using C = StageCfg<N, M, real, T, E>;
  using Tab = typename C::Tab;
  constexpr int Np = C::Np, Nm1p = C::Nm1p, Nfp = C::Nfp, Mp = C::Mp;
  constexpr int STRIDE = C::STRIDE, THREADS = C::THREADS;

  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  real* el = reinterpret_cast<real*>(smem + C::TAB);
  real* gs = el + E * STRIDE;
  real* c2s = gs + E * C::GEO;
  int* cs = reinterpret_cast<int*>(c2s + E * Mp);

  load_tables<C::TAB, THREADS>(smem, P.tables);

  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  const int64_t K = P.K;
  const size_t fs = size_t(K) * Np;  // field stride in global memory
  const int64_t ntiles = (K + E - 1) / E;
  bool bad = false;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * E;
    const int nE = int(K - e0 < E ? K - e0 : E);
    __syncthreads();  // tables ready / previous tile finished with shared memory

    // ---- stage the tile: q, geometry, c2, connectivity ----
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
      const real* src = P.qin + fld * fs + size_t(e0) * Np;
      for (int idx = threadIdx.x; idx < nE * Np; idx += THREADS) {
        const int e = idx / Np;
        el[e * STRIDE + fld * Np + (idx - e * Np)] = src[idx];
      }
    }
    for (int idx = threadIdx.x; idx < nE * 9; idx += THREADS) {
      const int e = idx / 9;
      gs[e * C::GEO + 3 + (idx - e * 9)] = P.geom[size_t(e0) * 9 + idx];
    }
    for (int idx = threadIdx.x; idx < nE * Mp; idx += THREADS) c2s[idx] = P.c2[size_t(e0) * Mp + idx];
    for (int idx = threadIdx.x; idx < nE * 4; idx += THREADS) cs[idx] = P.conn[size_t(e0) * 4 + idx];
    __syncthreads();
    // derived geometry: g_0 = -(g_1 + g_2 + g_3); face f: n = -g_f/|g_f|, |f|/|D| = 3 |g_f|
    for (int idx = threadIdx.x; idx < nE * 4; idx += THREADS) {
      const int e = idx >> 2, f = idx & 3;
      real* G = gs + e * C::GEO;
      real gx, gy, gz;
      if (f == 0) {
        gx = -(G[3] + G[6] + G[9]);
        gy = -(G[4] + G[7] + G[10]);
        gz = -(G[5] + G[8] + G[11]);
      } else {
        gx = G[3 * f];
        gy = G[3 * f + 1];
        gz = G[3 * f + 2];
      }
      const real gn = sqrt(gx * gx + gy * gy + gz * gz);
      const real inv = real(1) / gn;
      real* nr = G + 12 + 4 * f;
      nr[0] = -gx * inv;
      nr[1] = -gy * inv;
      nr[2] = -gz * inv;
      nr[3] = real(3) * gn;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nE; idx += THREADS) {
      real* G = gs + idx * C::GEO;
      G[0] = -(G[3] + G[6] + G[9]);
      G[1] = -(G[4] + G[7] + G[10]);
      G[2] = -(G[5] + G[8] + G[11]);
    }
    __syncthreads();

    const bool active = team < nE;
    const int e = active ? team : 0;
    real* Q = el + e * STRIDE;
    real* R = Q + 4 * Np;
    real* S = R + 4 * Np;
    const real* G = gs + e * C::GEO;
    real g[4][3];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int d = 0; d < 3; ++d) g[m][d] = G[3 * m + d];

    // ---- V1: barycentric combinations at degree N-1 ----
    for (int i = t; active && i < Nm1p; i += T) {
      int b0, j, k, l;
      unpack4(tab.dec3[off3(N - 1) + i], b0, j, k, l);
      const int im[4] = {idx3(N, j, k, l), idx3(N, j + 1, k, l), idx3(N, j, k + 1, l),
                         idx3(N, j, k, l + 1)};
      real gx = 0, gy = 0, gz = 0, dv = 0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const real p = Q[im[m]];
        gx += g[m][0] * p;
        gy += g[m][1] * p;
        gz += g[m][2] * p;
        dv += g[m][0] * Q[Np + im[m]] + g[m][1] * Q[2 * Np + im[m]] + g[m][2] * Q[3 * Np + im[m]];
      }
      S[i] = gx;
      S[Nm1p + i] = gy;
      S[2 * Nm1p + i] = gz;
      S[3 * Nm1p + i] = dv;
    }
    team_sync<T>();
    // ---- V2: elevate to degree N; rhs_u = -grad p, rhs_p = -div u ----
    for (int i = t; active && i < Np; i += T) {
      int a0, j, k, l;
      unpack4(tab.dec3[off3(N) + i], a0, j, k, l);
      real ax = 0, ay = 0, az = 0, ad = 0;
      auto add = [&](int s, int w) {
        const real wt = real(w);
        ax += wt * S[s];
        ay += wt * S[Nm1p + s];
        az += wt * S[2 * Nm1p + s];
        ad += wt * S[3 * Nm1p + s];
      };
      if (a0 > 0) add(idx3(N - 1, j, k, l), a0);
      if (j > 0) add(idx3(N - 1, j - 1, k, l), j);
      if (k > 0) add(idx3(N - 1, j, k - 1, l), k);
      if (l > 0) add(idx3(N - 1, j, k, l - 1), l);
      R[i] = -ad;
      R[Np + i] = -ax;
      R[2 * Np + i] = -ay;
      R[3 * Np + i] = -az;
    }
    team_sync<T>();

    // ---- F: penalty fluxes on the four faces, scaled by |f|/|D| ----
    real* Fp = S;
    real* Fu = S + 4 * Nfp;
    for (int it = t; active && it < 4 * Nfp; it += T) {
      const int f = it / Nfp;
      const int a = it - f * Nfp;
      const int io = tab.fidx[it];
      const real pm = Q[io], um = Q[Np + io], vm = Q[2 * Np + io], wm = Q[3 * Np + io];
      const int code = cs[e * 4 + f];
      real pp, up, vp, wp;
      if (code < 0) {  // p = 0 wall: mirror state
        pp = -pm;
        up = um;
        vp = vm;
        wp = wm;
      } else {
        const int64_t nb = int64_t(code >> 5);
        const int ni = tab.nidx[(((code >> 3) & 3) * 6 + (code & 7)) * Nfp + a];
        const int64_t loc = nb - e0;
        if (loc >= 0 && loc < nE) {
          const real* Qn = el + loc * STRIDE;
          pp = Qn[ni];
          up = Qn[Np + ni];
          vp = Qn[2 * Np + ni];
          wp = Qn[3 * Np + ni];
        } else {
          const real* qn = P.qin + size_t(nb) * Np + ni;
          pp = qn[0];
          up = qn[fs];
          vp = qn[2 * fs];
          wp = qn[3 * fs];
        }
      }
      const real* nr = G + 12 + 4 * f;
      const real jp = pp - pm;
      const real ndu = nr[0] * (up - um) + nr[1] * (vp - vm) + nr[2] * (wp - wm);
      const real hs = real(0.5) * nr[3];
      Fp[it] = hs * (P.tau_p * jp - ndu);
      Fu[it] = hs * (P.tau_u * ndu - jp);
    }
    team_sync<T>();

    // ---- L: lift L^f = E_L L0 per face, accumulated into rhs ----
    {
      real* bufA = S + 8 * Nfp;  // [p | u], Nfp each
      real* bufB = bufA + 2 * Nfp;
      const real third = real(1) / real(3);
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        const real* fp = Fp + f * Nfp;
        const real* fu = Fu + f * Nfp;
        const real* nr = G + 12 + 4 * f;
        const real nx = nr[0], ny = nr[1], nz = nr[2];
        // t = E'^T F at degree N-1 (integer weights b_x + 1)
        for (int i = t; active && i < np2(N - 1); i += T) {
          int b0, b1, b2, unused;
          unpack4(tab.dec2[off2(N - 1) + i], b0, b1, b2, unused);
          const int i0 = idx2(N, b1, b2), i1 = idx2(N, b1 + 1, b2), i2 = idx2(N, b1, b2 + 1);
          bufB[i] = real(b0 + 1) * fp[i0] + real(b1 + 1) * fp[i1] + real(b2 + 1) * fp[i2];
          bufB[Nfp + i] = real(b0 + 1) * fu[i0] + real(b1 + 1) * fu[i1] + real(b2 + 1) * fu[i2];
        }
        team_sync<T>();
        // g0 = L0 F = ((2N+3) F + E' t) / 3; layer 0 (ell_0 = 1)
        for (int i = t; active && i < Nfp; i += T) {
          int a0, a1, a2, unused;
          unpack4(tab.dec2[off2(N) + i], a0, a1, a2, unused);
          real ep = 0, eu = 0;
          if (a0 > 0) {
            const int s = idx2(N - 1, a1, a2);
            ep += real(a0) * bufB[s];
            eu += real(a0) * bufB[Nfp + s];
          }
          if (a1 > 0) {
            const int s = idx2(N - 1, a1 - 1, a2);
            ep += real(a1) * bufB[s];
            eu += real(a1) * bufB[Nfp + s];
          }
          if (a2 > 0) {
            const int s = idx2(N - 1, a1, a2 - 1);
            ep += real(a2) * bufB[s];
            eu += real(a2) * bufB[Nfp + s];
          }
          const real gp = (real(2 * N + 3) * fp[i] + ep) * third;
          const real gu = (real(2 * N + 3) * fu[i] + eu) * third;
          bufA[i] = gp;
          bufA[Nfp + i] = gu;
          const int vi = tab.lidx[f * Np + i];
          R[vi] += gp;
          R[Np + vi] += nx * gu;
          R[2 * Np + vi] += ny * gu;
          R[3 * Np + vi] += nz * gu;
        }
        team_sync<T>();
        real* cur = bufA;
        real* nxt = bufB;
        int off = Nfp;
#pragma unroll 1
        for (int layer = 1; layer <= N; ++layer) {
          const int n2 = N - layer;
          const real inv = real(1) / real(n2 + 1);
          const real ell = tab.ell[layer];
          for (int i = t; active && i < np2(n2); i += T) {
            int b0, b1, b2, unused;
            unpack4(tab.dec2[off2(n2) + i], b0, b1, b2, unused);
            const int i0 = idx2(n2 + 1, b1, b2), i1 = idx2(n2 + 1, b1 + 1, b2),
                      i2 = idx2(n2 + 1, b1, b2 + 1);
            const real gp =
                (real(b0 + 1) * cur[i0] + real(b1 + 1) * cur[i1] + real(b2 + 1) * cur[i2]) * inv;
            const real gu = (real(b0 + 1) * cur[Nfp + i0] + real(b1 + 1) * cur[Nfp + i1] +
                             real(b2 + 1) * cur[Nfp + i2]) *
                            inv;
            nxt[i] = gp;
            nxt[Nfp + i] = gu;
            const int vi = tab.lidx[f * Np + off + i];
            R[vi] += ell * gp;
            const real eu = ell * gu;
            R[Np + vi] += nx * eu;
            R[2 * Np + vi] += ny * eu;
            R[3 * Np + vi] += nz * eu;
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
      real* B = S + C::BUF;
      const bool is_src = active && (e0 + e == P.src_elem);
      for (int i = t; active && i < Np; i += T) {
        real v = R[i];
        if (is_src) v += P.src_amp * P.src_vec[i];
        A[i] = v * tab.invfactN[i];
      }
      if (active && t == 0) A[Np] = real(0);
      real bh[Mp > 0 ? Mp : 1];
#pragma unroll
      for (int b = 0; b < Mp; ++b) bh[b] = c2s[e * Mp + b] * tab.invfactM[b];
      team_sync<T>();
      real lv[N + 1][C::RMAX];
      wadg_element<N, M, real, T, C::RMAX>(tab, A, B, bh, active, t, lv);
#pragma unroll
      for (int r = 0; r < C::RMAX; ++r) {
        const int i = t + r * T;
        if (active && i < Np) R[i] = lv[0][r];
      }
    }
    __syncthreads();

    // ---- RK: res = a res + dt rhs; q_out = q_in + b res (coalesced over the tile) ----
    const bool read_res = P.a != real(0);
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) {
      const size_t base = fld * fs + size_t(e0) * Np;
      for (int idx = threadIdx.x; idx < nE * Np; idx += THREADS) {
        const int ee = idx / Np;
        const int i = idx - ee * Np;
        const real rhs = el[ee * STRIDE + 4 * Np + fld * Np + i];
        const real q = el[ee * STRIDE + fld * Np + i];
        real r = P.dt * rhs;
        if (read_res) r += P.a * P.res[base + idx];
        P.res[base + idx] = r;
        const real qn = q + P.b * r;
        P.qout[base + idx] = qn;
        bad |= !isfinite(qn);
      }
    }
  }
  if (bad) atomicOr(P.status, 1u);
}

// The weight-adjusted update alone: out = P^{N+M}_N (c2 * rhs) per element.
template <int N, int M, typename real, int T, int E>
__global__ void __launch_bounds__(T* E) wadg_kernel(const WadgParams<real> P) {
  using C = StageCfg<N, M, real, T, E>;
  using Tab = typename C::Tab;
  constexpr int Np = C::Np, Mp = C::Mp, STRIDE = C::STRIDE, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  real* el = reinterpret_cast<real*>(smem + C::TAB);
  real* c2s = el + E * STRIDE;
  load_tables<C::TAB, THREADS>(smem, P.tables);
  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  const int64_t ntiles = (P.K + E - 1) / E;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * E;
    const int nE = int(P.K - e0 < E ? P.K - e0 : E);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nE * Np; idx += THREADS) {
      const int e = idx / Np;
      el[e * STRIDE + (idx - e * Np)] = P.rhs[size_t(e0) * Np + idx];
    }
    for (int idx = threadIdx.x; idx < nE * Mp; idx += THREADS) c2s[idx] = P.c2[size_t(e0) * Mp + idx];
    __syncthreads();
    const bool active = team < nE;
    const int e = active ? team : 0;
    real* R = el + e * STRIDE;
    real* A = R + Np;
    real* B = A + C::BUF;
    for (int i = t; active && i < Np; i += T) A[i] = R[i] * tab.invfactN[i];
    if (active && t == 0) A[Np] = real(0);
    real bh[Mp > 0 ? Mp : 1];
#pragma unroll
    for (int b = 0; b < Mp; ++b) bh[b] = c2s[e * Mp + b] * tab.invfactM[b];
    team_sync<T>();
    real lv[N + 1][C::RMAX];
    wadg_element<N, M, real, T, C::RMAX>(tab, A, B, bh, active, t, lv);
#pragma unroll
    for (int r = 0; r < C::RMAX; ++r) {
      const int i = t + r * T;
      if (active && i < Np) R[i] = lv[0][r];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nE * Np; idx += THREADS) {
      const int e2 = idx / Np;
      P.out[size_t(e0) * Np + idx] = el[e2 * STRIDE + (idx - e2 * Np)];
    }
  }
}

}  // namespace bbw
