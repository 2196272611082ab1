// bbw_elastic.cuh -- fused BBWADG elastic LSRK stage for sm_103a.
//
// One launch runs one stage of the five-stage low-storage RK4 for the
// velocity-stress elastic system of Sec. 2.2 (Eq. ewave) over all elements:
// nine fields per element, v = (v_x, v_y, v_z) and the six unique stress
// entries s = (s_xx, s_yy, s_zz, s_yz, s_xz, s_xy), with the matrix-weighted
// update of Eq. (ewadg) applied as scalar weight-adjusted projections.
//
// The work decomposition is that of the acoustic stage kernel (groups of V
// interleaved elements, teams of T lanes, operator tables once per CTA,
// gather stencils driven by packed table words); the Bernstein operators and
// the projection P~_N are the same device code. Per group and stage:
//   F1  neighbour traces of the nine fields on the four faces (cp.async from
//       q_in in L2), in flight while
//   V1  the degree N-1 barycentric combinations of Sec. 4 give, per node,
//       sum_i A_i^T d s/dx_i (3 rows) and sum_i A_i d v/dx_i (6 rows);
//   F2  penalty fluxes ([[x]] = x+ - x, A_n = sum_i n_i A_i):
//         F_v = (1/2) A_n^T [[s]] + (tau_v/2) A_n^T A_n [[v]]
//         F_s = A_n h,  h = (1/2) [[v]] + (tau_s/2) A_n^T [[s]]
//       (A_n is constant on an affine face, so h is lifted and A_n applied
//       after the lift: six lifted quantities per face instead of nine);
//   L   per face the lift pyramids of the six quantities (L^f = E_L L0);
//   V2  per node one degree elevation of V1 plus the four face
//       contributions, into the right-hand side R [9][Np];
//   W   weight-adjusted update: v_c <- P(rho^{-1} R_v,c); for the stress
//       P(lambda tr R_s) once, then s_a <- P(mu 2 R_s,a) + P(lambda tr R_s)
//       for the normal entries and P(mu R_s,a) for the shear entries (the
//       isotropic C of Sec. 2.2), each P the product of Sec. 5.1 followed by
//       the projection of Eq. (20); then the RK update of that field.
// Walls are traction-free mirrors: s+ = -s, v+ = v.
#pragma once

#include "bbw_stage.cuh"

namespace bbw {

template <typename real>
struct ElasticParams {
  const real* __restrict__ qin;   // [G][9][Np][V]
  real* __restrict__ qout;        // [G][9][Np][V]
  real* __restrict__ res;         // [G][9][Np][V], updated in place
  const real* __restrict__ media;  // [G][3][Mp][V]: rho^{-1}, lambda, mu
  const real* __restrict__ geom;  // [G][9][V]: d lambda_m / d x_i, m = 1..3
  const int32_t* __restrict__ conn;  // [G][4][V] packed neighbour words
  const void* __restrict__ tables;   // Tables<N, M, real>
  int64_t G;
  real a, b, dt;
  real tau_v, tau_s;
  unsigned int* status;  // bit 0: non-finite output; bit 1 (checked build): index out of range
};

template <int N, typename real>
struct ElasticShape;
template <int N>
struct ElasticShape<N, float> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : N <= 7 ? 32 : 64;
  static constexpr int V = N <= 5 ? 2 : 1;
};
template <int N>
struct ElasticShape<N, double> {
  static constexpr int T = N == 1 ? 4 : N == 2 ? 8 : N == 3 ? 16 : N <= 7 ? 32 : 64;
  static constexpr int V = 1;
};

template <int N, int M, typename real, int T, int V, int GC>
struct ElasticCfg {
  static constexpr int Np = np3(N);
  static constexpr int Nm1p = np3(N - 1);
  static constexpr int Nfp = np2(N);
  static constexpr int Mp = np3(M);
  static constexpr int NMp = np3(N + M);
  static constexpr int THREADS = T * GC;
  static constexpr int BUF = NMp > Np + 1 ? NMp : Np + 1;
  // per-team region, in vectors of V:
  //   Q [9][Np] | PYR [6][4][Np] | V1B [9][Nm1p] | TR [9][4][Nfp] (N < 5) |
  //   normals [4][4] | media [3][Mp] | connectivity words [4][V] (int32)
  // From N = 5 the neighbour traces fit the pyramid blocks above level 0
  // (6 (Np - Nfp) >= 9 Nfp), which stay free until F2 has read them; below,
  // they have a region of their own. The right-hand side R [9][Np] reuses Q
  // once F2 has read the own traces (the RK update reads q_in from global
  // memory, an L2 hit). The WADG ping-pong buffers reuse PYR after V2.
  static constexpr bool TR_IN_P = 6 * (Np - Nfp) >= 9 * Nfp;
  // FP32 projects the fields in pairs (vectors of 2V, 16-byte aligned
  // ping-pong buffers in the pyramid region); FP64 one field at a time
  static constexpr bool PAIR = sizeof(real) == 4;
  static constexpr int S_W = PAIR ? 4 * BUF + 4 : 2 * BUF;
  static constexpr int S_PYR = 24 * Np > S_W ? 24 * Np : S_W;
  static constexpr int S_V1 = 9 * Nm1p;
  static constexpr int S_TR = TR_IN_P ? 0 : 36 * Nfp;
  static constexpr int CONNV = (16 * V + int(sizeof(real)) * V - 1) / (int(sizeof(real)) * V);  // 4 V int32
  static constexpr int TEAMV = (9 * Np + S_PYR + S_V1 + S_TR + 16 + 3 * Mp + CONNV) | 1;
  static constexpr int TAB = table_bytes<N, M, real>();
  static constexpr int SMEM = TAB + int(sizeof(real)) * V * GC * TEAMV;
  static_assert(SMEM <= kSmemPerCta, "shared memory of the launch shape");
  static constexpr int RMAX = (Np + T - 1) / T;
  static_assert(T >= 4 && (T <= 32 ? 32 % T == 0 : T % 32 == 0), "team: a divisor or a multiple of a warp");
  static_assert(T <= 32 || GC <= 15, "one named barrier per multi-warp team");
};

// Thread budget of one CTA: 128 below N = 4 (several CTAs per SM), else one
// CTA per SM with up to 512 threads. The paired projections with V = 2 keep
// 4-wide telescoping levels in registers: at N = 4 they fit 384 threads, at
// N = 5 256 (ptxas: no spills at M <= 2).
template <int N, int V, typename real>
constexpr int elastic_cta_threads() {
  if (N <= 3) return 128;
  if (V > 1 && sizeof(real) == 4) return N == 4 ? 384 : 256;
  return 512;
}

// Teams per CTA: as many as fit the shared memory and the thread budget.
template <int N, int M, typename real, int T, int V>
constexpr int elastic_cta_groups() {
  constexpr int team_bytes = int(sizeof(real)) * V * ElasticCfg<N, M, real, T, V, 1>::TEAMV;
  constexpr int by_smem = (kSmemPerCta - table_bytes<N, M, real>()) / team_bytes;
  constexpr int by_threads = elastic_cta_threads<N, V, real>() / T;
  constexpr int g = by_smem < by_threads ? by_smem : by_threads;
  return T > 32 && g > 15 ? 15 : g;
}

// traction A_n^T s of a stress vector (xx, yy, zz, yz, xz, xy)
template <typename real, int V>
__device__ __forceinline__ void traction(const vec<real, V>& n0, const vec<real, V>& n1, const vec<real, V>& n2,
                                         const vec<real, V> (&s)[6], vec<real, V> (&t)[3]) {
  t[0] = vmul(n0, s[0]);
  vfma(t[0], n1, s[5]);
  vfma(t[0], n2, s[4]);
  t[1] = vmul(n0, s[5]);
  vfma(t[1], n1, s[1]);
  vfma(t[1], n2, s[3]);
  t[2] = vmul(n0, s[4]);
  vfma(t[2], n1, s[3]);
  vfma(t[2], n2, s[2]);
}
// A_n v: the symmetric product of n and v in the same order
template <typename real, int V>
__device__ __forceinline__ void sym_normal(const vec<real, V>& n0, const vec<real, V>& n1, const vec<real, V>& n2,
                                           const vec<real, V> (&v)[3], vec<real, V> (&s)[6]) {
  s[0] = vmul(n0, v[0]);
  s[1] = vmul(n1, v[1]);
  s[2] = vmul(n2, v[2]);
  s[3] = vmul(n2, v[1]);
  vfma(s[3], n1, v[2]);
  s[4] = vmul(n2, v[0]);
  vfma(s[4], n0, v[2]);
  s[5] = vmul(n1, v[0]);
  vfma(s[5], n0, v[1]);
}

template <int N, int M, typename real, int T, int V, int GC>
__global__ void __launch_bounds__(T* GC) elastic_stage_kernel(const ElasticParams<real> P) {
  using C = ElasticCfg<N, M, real, T, V, GC>;
  using Tab = Tables<N, M, real>;
  using vt = vec<real, V>;
  constexpr int Np = C::Np, Nm1p = C::Nm1p, Nfp = C::Nfp, Mp = C::Mp;
  constexpr int QV = 9 * Np;

  extern __shared__ __align__(16) unsigned char smem[];
  const Tab& tab = *reinterpret_cast<const Tab*>(smem);
  load_tables<C::TAB, C::THREADS>(smem, P.tables);
  __syncthreads();

  const int team = threadIdx.x / T;
  const int t = threadIdx.x % T;
  real* Q = reinterpret_cast<real*>(smem + C::TAB) + team * C::TEAMV * V;  // [9][Np]
  real* PYR = Q + QV * V;                 // [6][4][Np]
  real* V1B = PYR + C::S_PYR * V;         // [9][Nm1p]
  real* TR = V1B + C::S_V1 * V;           // [9][4][Nfp] (N < 5)
  real* NRM = TR + C::S_TR * V;           // [4][nx, ny, nz, (1/2)|f|/|D|]
  real* MED = NRM + 16 * V;               // [3][Mp]
  int* CS = reinterpret_cast<int*>(MED + 3 * Mp * V);  // [4][V]
  auto pyr = [&](int k, int f, int slot) { return PYR + ((k * 4 + f) * Np + slot) * V; };
  // neighbour trace of field fld at face node a of face f
  auto trace = [&](int fld, int f, int a) -> real* {
    if constexpr (C::TR_IN_P) {
      constexpr int FREE = Np - Nfp;  // slots above level 0 in one pyramid block
      const int j = fld * Nfp + a;
      const int k = j / FREE;
      return pyr(k, f, Nfp + (j - k * FREE));
    } else {
      return TR + ((fld * 4 + f) * Nfp + a) * V;
    }
  };
  real* R = Q;  // [9][Np] right-hand side, written in V2 (Q is not read after F2)

  const int64_t G = P.G;
  const int64_t stride = int64_t(gridDim.x) * GC;
  const bool read_res = P.a != real(0);
  bool bad = false;
  bool oob = false;
  (void)oob;

  for (int64_t g = int64_t(blockIdx.x) * GC + team; g < G; g += stride) {
    if (t == 0 && g + stride < G) {
      const size_t qb = size_t(QV) * V * sizeof(real);
      prefetch_l2(P.qin + size_t(g + stride) * QV * V, uint32_t(qb));
      if (read_res) prefetch_l2(P.res + size_t(g + stride) * QV * V, uint32_t(qb));
    }
    {
      constexpr int VB = V * int(sizeof(real));
      const real* qg = P.qin + size_t(g) * QV * V;
      for (int idx = t; idx < QV; idx += T) cp_async<VB>(Q + idx * V, qg + size_t(idx) * V);
      for (int idx = t; idx < 3 * Mp; idx += T)
        cp_async<VB>(MED + idx * V, P.media + (size_t(g) * 3 * Mp + idx) * V);
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

    // ---- F1: neighbour traces of the nine fields ----
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
          for (int fld = 0; fld < 9; ++fld) cp_async<int(sizeof(real))>(trace(fld, f, a) + v, src + fld * Np * V);
        }
      }
    }

    // ---- V1: degree N-1 combinations. Rows 0..2: sum_i A_i^T d s/dx_i;
    // rows 3..8: sum_i A_i d v/dx_i (strain rate, engineering shear) ----
    for (int i = t; i < Nm1p; i += T) {
      const Stencil3 s = unpack_stencil3(tab.red3[off3(N - 1) + i]);
      const int im[4] = {s.base, s.base + 1, s.base + s.dk, s.base + s.dl};
      vt o[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) o[k] = vzero<real, V>();
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const vt gx = gm[m][0], gy = gm[m][1], gz = gm[m][2];
        const vt v0 = vld<real, V>(Q + im[m] * V), v1 = vld<real, V>(Q + (Np + im[m]) * V),
                 v2 = vld<real, V>(Q + (2 * Np + im[m]) * V);
        const vt sxx = vld<real, V>(Q + (3 * Np + im[m]) * V), syy = vld<real, V>(Q + (4 * Np + im[m]) * V),
                 szz = vld<real, V>(Q + (5 * Np + im[m]) * V), syz = vld<real, V>(Q + (6 * Np + im[m]) * V),
                 sxz = vld<real, V>(Q + (7 * Np + im[m]) * V), sxy = vld<real, V>(Q + (8 * Np + im[m]) * V);
        vfma(o[0], gx, sxx);
        vfma(o[0], gy, sxy);
        vfma(o[0], gz, sxz);
        vfma(o[1], gx, sxy);
        vfma(o[1], gy, syy);
        vfma(o[1], gz, syz);
        vfma(o[2], gx, sxz);
        vfma(o[2], gy, syz);
        vfma(o[2], gz, szz);
        vfma(o[3], gx, v0);
        vfma(o[4], gy, v1);
        vfma(o[5], gz, v2);
        vfma(o[6], gz, v1);
        vfma(o[6], gy, v2);
        vfma(o[7], gz, v0);
        vfma(o[7], gx, v2);
        vfma(o[8], gy, v0);
        vfma(o[8], gx, v1);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) vst(V1B + (k * Nm1p + i) * V, o[k]);
    }
    cp_async_wait_all();
    team_sync<T>();

    // ---- F2: fluxes into level 0 of the pyramids: k = 0..2 F_v, k = 3..5 h ----
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
      vt jv[3], js[6];
#pragma unroll
      for (int fld = 0; fld < 9; ++fld) {
        const vt own = vld<real, V>(Q + (fld * Np + io) * V);
        vt nbv = vld<real, V>(trace(fld, f, a));
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (CS[f * V + v] < 0) nbv.set(v, fld < 3 ? own.get(v) : -own.get(v));  // traction-free mirror
        if (fld < 3)
          jv[fld] = vsub(nbv, own);
        else
          js[fld - 3] = vsub(nbv, own);
      }
      const vt n0 = vld<real, V>(NRM + (4 * f + 0) * V), n1 = vld<real, V>(NRM + (4 * f + 1) * V),
               n2 = vld<real, V>(NRM + (4 * f + 2) * V), hs = vld<real, V>(NRM + (4 * f + 3) * V);
      vt ts[3], anv[6], tan[3];
      traction(n0, n1, n2, js, ts);
      sym_normal(n0, n1, n2, jv, anv);
      traction(n0, n1, n2, anv, tan);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        vst(pyr(c, f, a), vmul(hs, vaxpy(ts[c], P.tau_v, tan[c])));
        vst(pyr(3 + c, f, a), vmul(hs, vaxpy(jv[c], P.tau_s, ts[c])));
      }
    }
    team_sync<T>();

    // ---- L: lift pyramids of the six quantities of the four faces ----
    {
      constexpr int CT = np2(N - 1);
      for (int it = t; it < 4 * CT; it += T) {
        const int f = it / CT;
        const int i = it - f * CT;
        const Stencil2 s = unpack_stencil2(tab.red2[off2(N - 1) + i]);
        const real w0 = real(N + 2 - s.w1 - s.w2), w1 = real(s.w1), w2 = real(s.w2);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          vt x = vmuls(w0, vld<real, V>(pyr(k, f, s.base)));
          vfmas(x, w1, vld<real, V>(pyr(k, f, s.base + 1)));
          vfmas(x, w2, vld<real, V>(pyr(k, f, s.base + s.db)));
          vst(pyr(k, f, Nfp + i), x);
        }
      }
      team_sync<T>();
      const real third = real(1) / real(3);
      for (int it = t; it < 4 * Nfp; it += T) {
        const int f = it / Nfp;
        const int i = it - f * Nfp;
        const Stencil2 s = unpack_stencil2(tab.elev2[i]);
        const int a0 = N - s.w1 - s.w2;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          vt x = vmuls(real(2 * N + 3), vld<real, V>(pyr(k, f, i)));
          if (a0 > 0) vfmas(x, real(a0), vld<real, V>(pyr(k, f, Nfp + s.base)));
          if (s.w1 > 0) vfmas(x, real(s.w1), vld<real, V>(pyr(k, f, Nfp + s.base - 1)));
          if (s.w2 > 0) vfmas(x, real(s.w2), vld<real, V>(pyr(k, f, Nfp + s.base - s.db)));
          vst(pyr(k, f, i), vmuls(third, x));
        }
      }
      team_sync<T>();
#pragma unroll 1
      for (int lv = 1; lv <= N; ++lv) {
        const int n2 = N - lv;
        const int cnt = np2(n2);
        const int src = lift_level_base(N, lv - 1), dst = lift_level_base(N, lv);
        const real icnt = real(1) / real(cnt);
        const real scale = tab.lscale[lv];
        for (int it = t; it < 4 * cnt; it += T) {
          const int f = int((real(it) + real(0.5)) * icnt);
          const int i = it - f * cnt;
          const Stencil2 s = unpack_stencil2(tab.red2[off2(n2) + i]);
          const real w0 = real(n2 + 3 - s.w1 - s.w2) * scale, w1 = real(s.w1) * scale, w2 = real(s.w2) * scale;
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            vt x = vmuls(w0, vld<real, V>(pyr(k, f, src + s.base)));
            vfmas(x, w1, vld<real, V>(pyr(k, f, src + s.base + 1)));
            vfmas(x, w2, vld<real, V>(pyr(k, f, src + s.base + s.db)));
            vst(pyr(k, f, dst + i), x);
          }
        }
        team_sync<T>();
      }
    }

    // ---- V2 + lift gather: R = E V1 + sum_f (F_v ; A_n h) lifted ----
    {
      vt nrm[4][3];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int d = 0; d < 3; ++d) nrm[f][d] = vld<real, V>(NRM + (4 * f + d) * V);
      for (int i = t; i < Np; i += T) {
        const Stencil3 s = unpack_stencil3(tab.elev3[off3(N) + i]);
        const int a0 = N - s.w1 - s.w2 - s.w3;
        vt r[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) r[k] = vzero<real, V>();
        auto add = [&](int idx, int w) {
          const real wt = real(w);
#pragma unroll
          for (int k = 0; k < 9; ++k) vfmas(r[k], wt, vld<real, V>(V1B + (k * Nm1p + idx) * V));
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
          vt h[3], an[6];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            r[c] = vaxpy(r[c], real(1), vld<real, V>(pyr(c, f, o)));
            h[c] = vld<real, V>(pyr(3 + c, f, o));
          }
          sym_normal(nrm[f][0], nrm[f][1], nrm[f][2], h, an);
#pragma unroll
          for (int k = 0; k < 6; ++k) r[3 + k] = vaxpy(r[3 + k], real(1), an[k]);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) vst(R + (k * Np + i) * V, r[k]);
      }
    }
    team_sync<T>();

    // ---- W + RK: weight-adjusted update of every field, then its RK update ----
    {
      real* resg = P.res + size_t(g) * QV * V;
      real* qog = P.qout + size_t(g) * QV * V;
      vt ptr[C::RMAX];  // P(lambda tr R_s)
      const real* qig = P.qin + size_t(g) * QV * V;
      // res and q_in of field fld at this lane's nodes, loaded before the
      // field's projection so that the loads are in flight during it
      vt pres[2][C::RMAX], pq[2][C::RMAX];
      auto prefetch = [&](int slot, int fld) {
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) {
          const int i = t + r * T;
          const bool ok = i < Np;
          pres[slot][r] = ok && read_res ? vld<real, V>(resg + size_t(fld * Np + i) * V) : vzero<real, V>();
          pq[slot][r] = ok ? vld<real, V>(qig + size_t(fld * Np + i) * V) : vzero<real, V>();
        }
      };
      // RK update of field fld from its weight-adjusted right-hand side
      auto rk1 = [&](int fld, int slot, int r, vt rhs) {
        const int i = t + r * T;
        vt rn = vmuls(P.dt, rhs);
        vfmas(rn, P.a, pres[slot][r]);
        vst(resg + size_t(fld * Np + i) * V, rn);
        const vt qn = vaxpy(pq[slot][r], P.b, rn);
        vst(qog + size_t(fld * Np + i) * V, qn);
#pragma unroll
        for (int v = 0; v < V; ++v) bad |= !isfinite(qn.get(v));
      };
      // (sum of the fields R[k], k in [k0, k0 + nk)) * wt / alpha! at node i
      auto rsum = [&](int k0, int nk, real wt, int i) {
        vt x = vld<real, V>(R + (k0 * Np + i) * V);
        for (int k = 1; k < nk; ++k) x = vaxpy(x, real(1), vld<real, V>(R + ((k0 + k) * Np + i) * V));
        return vmuls(wt * tab.invfactN[i], x);
      };
      if constexpr (C::PAIR) {
        // two fields per projection: vectors of 2V lanes (the first field's
        // V element lanes, then the second's), each lane with its own weight
        constexpr int W2 = 2 * V;
        using wt2 = vec<real, W2>;
        real* A2 = reinterpret_cast<real*>((reinterpret_cast<uintptr_t>(PYR) + 15) & ~uintptr_t(15));
        real* B2 = A2 + C::BUF * W2;
        wt2 lv[N + 1][C::RMAX];
        // project (wt1 sum R[k1..k1+n1) ; wt2 sum R[k2..k2+n2)) with weights (w1 ; w2)
        auto project = [&](int k1, int n1, real s1, int w1, int k2, int n2, real s2, int w2) {
          for (int i = t; i < Np; i += T) {
            vst<real, V>(A2 + i * W2, rsum(k1, n1, s1, i));
            vst<real, V>(A2 + i * W2 + V, rsum(k2, n2, s2, i));
          }
          if (t == 0) vst<real, W2>(A2 + Np * W2, vzero<real, W2>());
          wt2 bh2[Mp];  // weight coefficients / beta!, per lane
#pragma unroll
          for (int b = 0; b < Mp; ++b)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              bh2[b].set(v, tab.invfactM[b] * MED[(w1 * Mp + b) * V + v]);
              bh2[b].set(V + v, tab.invfactM[b] * MED[(w2 * Mp + b) * V + v]);
            }
          team_sync<T>();
          wadg_group<N, M, real, T, W2, C::RMAX>(tab, A2, B2, bh2, true, t, lv);
        };
        auto half = [&](const wt2& x, int h) {
          vt y;
#pragma unroll
          for (int v = 0; v < V; ++v) y.set(v, x.get(h * V + v));
          return y;
        };
        // (v_x, v_y) with rho^{-1}
        prefetch(0, 0);
        prefetch(1, 1);
        project(0, 1, real(1), 0, 1, 1, real(1), 0);
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r)
          if (t + r * T < Np) {
            rk1(0, 0, r, half(lv[0][r], 0));
            rk1(1, 1, r, half(lv[0][r], 1));
          }
        // (v_z with rho^{-1}, tr R_s with lambda)
        prefetch(0, 2);
        project(2, 1, real(1), 0, 3, 3, real(1), 1);
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r)
          if (t + r * T < Np) {
            rk1(2, 0, r, half(lv[0][r], 0));
            ptr[r] = half(lv[0][r], 1);
          }
        // (s_xx, s_yy) with mu, times 2, plus P(lambda tr)
        prefetch(0, 3);
        prefetch(1, 4);
        project(3, 1, real(2), 2, 4, 1, real(2), 2);
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r)
          if (t + r * T < Np) {
            rk1(3, 0, r, vaxpy(half(lv[0][r], 0), real(1), ptr[r]));
            rk1(4, 1, r, vaxpy(half(lv[0][r], 1), real(1), ptr[r]));
          }
        // (s_zz with 2 mu plus P(lambda tr), s_yz with mu)
        prefetch(0, 5);
        prefetch(1, 6);
        project(5, 1, real(2), 2, 6, 1, real(1), 2);
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r)
          if (t + r * T < Np) {
            rk1(5, 0, r, vaxpy(half(lv[0][r], 0), real(1), ptr[r]));
            rk1(6, 1, r, half(lv[0][r], 1));
          }
        // (s_xz, s_xy) with mu
        prefetch(0, 7);
        prefetch(1, 8);
        project(7, 1, real(1), 2, 8, 1, real(1), 2);
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r)
          if (t + r * T < Np) {
            rk1(7, 0, r, half(lv[0][r], 0));
            rk1(8, 1, r, half(lv[0][r], 1));
          }
      } else {
        real* A = PYR;
        real* B = PYR + C::BUF * V;
        vt bh[3][Mp];  // weight coefficients / beta!
#pragma unroll
        for (int w = 0; w < 3; ++w)
#pragma unroll
          for (int b = 0; b < Mp; ++b) bh[w][b] = vmuls(tab.invfactM[b], vld<real, V>(MED + (w * Mp + b) * V));
        vt lv[N + 1][C::RMAX];
        auto project = [&](int k0, int nk, real wt, int w) {
          for (int i = t; i < Np; i += T) vst(A + i * V, rsum(k0, nk, wt, i));
          if (t == 0) vst(A + Np * V, vzero<real, V>());
          team_sync<T>();
          wadg_group<N, M, real, T, V, C::RMAX>(tab, A, B, bh[w], true, t, lv);
        };
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {  // velocity: rho^{-1}
          prefetch(0, c);
          project(c, 1, real(1), 0);
#pragma unroll
          for (int r = 0; r < C::RMAX; ++r)
            if (t + r * T < Np) rk1(c, 0, r, lv[0][r]);
        }
        project(3, 3, real(1), 1);  // lambda tr(R_s)
#pragma unroll
        for (int r = 0; r < C::RMAX; ++r) ptr[r] = lv[0][r];
#pragma unroll 1
        for (int a = 0; a < 6; ++a) {  // mu: 2 R_s,a on the normal entries, R_s,a on the shear entries
          prefetch(0, 3 + a);
          project(3 + a, 1, a < 3 ? real(2) : real(1), 2);
#pragma unroll
          for (int r = 0; r < C::RMAX; ++r)
            if (t + r * T < Np) rk1(3 + a, 0, r, a < 3 ? vaxpy(lv[0][r], real(1), ptr[r]) : lv[0][r]);
        }
      }
    }
    team_sync<T>();
  }
  if (bad) atomicOr(P.status, 1u);
  if constexpr (kChecked) {
    if (oob) atomicOr(P.status, 2u);
  }
}

}  // namespace bbw
