// bbw_adjoint.cu -- receivers, recorded forward runs and the discrete adjoint
// of the LSRK time stepping with respect to the c^2 coefficients.
//
// The semi-discrete system is dq/dt = L q + s(t) with L = M_w^{-1} K(tau):
// M_w = blockdiag(|D| M (M_{c2})^{-1} M, |D| M, |D| M, |D| M) per element
// (the weight-adjusted mass of Eq. (4): its inverse applied to the pressure
// is |D|^{-1} P~(c^2 . M^{-1} .), Sec. 5), and K(tau) the DG stiffness and
// flux matrix of Eq. (2). The central-flux part of K is skew and the penalty
// part symmetric and linear in (tau_p, tau_u) (the energy argument of the
// method), so K(tau)^T = -K(-tau) and
//
//     L(tau)^T r = -M_w L(-tau) M_w^{-1} r = -|D| M A_{-tau}(y),
//     y = [ |D|^{-1} P~(c^2 . M^{-1} r_p) ; |D|^{-1} M^{-1} r_u ],
//
// A_{-tau} being the stage kernel's spatial operator (volume terms plus lifted
// fluxes, before the weight-adjusted update) with negated penalties.
//
// Adjoint of one LSRK stage s (res' = a_s res + dt (L q + s), q' = q + b_s res'),
// from the cotangents (qbar, rbar) of (q', res'):
//     rt = rbar + b_s qbar;   qbar += dt L^T rt;   rbar = a_s rt;
//     gc2[k][beta] += dt (M^{-1} rt_p)_k^T T_beta v_k,
// with T_beta the mass matrix weighted by the degree-M Bernstein polynomial
// beta and v = (A_tau q + source)_p the pressure bracket of the forward stage.
//
// Dual variables. With kap = M^{-1} qbar and rho = M^{-1} rbar per element and
// field (M the reference mass matrix), the recursion has no mass matrix left:
//     rho_t = a rho + b_s kap,   y = [P~(c^2 rho_t,p) ; rho_t,u] / |D|,
//     kap  -= dt |D| A_{-tau}(y),  gc2[k][beta] += dt rho_t,p^T T_beta v,
// receivers inject M^{-1} B(x_r) (their dual vectors, computed once on the
// host) and the state gradient is M kap at the end. One adjoint stage is three
// launches of this library's kernels: the pre-kernel (rho_t and y, with the
// weight-adjusted update of the forward kernel), the spatial kernel in its
// accumulate mode (kap -= dt |D| A_{-tau}(y)), and the c^2 gradient kernel.
//
// The gradient term: rho^T T_beta v = int rho v B_beta over the reference
// element = C_b sum_gamma w_gamma (gamma + beta)! / beta!, with
// w_gamma = sum_{alpha + alpha' = gamma} (rho_alpha / alpha!) (v_alpha' / alpha'!)
// the factorial-scaled Bernstein product of rho and v (degree 2N, Sec. 5.1)
// and C_b = 6 (N!)^2 M! / (2N+M+3)! (Dirichlet moments).
//
// A recorded run keeps the state every C steps (checkpoints) and the step
// counter of every step; the backward pass recomputes one checkpoint segment
// at a time with the forward stage kernel, which stores the pressure bracket
// of each stage (memory: the checkpoints plus 5 C pressure fields).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bbw_common.h"
#include "bbw_ops.h"
#include "bbw_solver.h"
#include "bbw_stage.cuh"
#include "bbwadg.h"

using bbw::fail;

// warps per block of the c^2 gradient kernel
constexpr int kGradWarps = 8;
constexpr int kMaxMp = 20;

struct AdjointData {
  // receivers: element, Bernstein basis values B_i(lambda(x_r)) [nrec][Np]
  // (sampling) and their dual vectors M^{-1} B(x_r) (adjoint injection)
  int64_t nrec = 0;
  std::vector<int64_t> rec_elem;
  int64_t* d_rec_elem = nullptr;
  void* d_rec_vec = nullptr;
  void* d_rec_dual = nullptr;
  // the receivers grouped by element (internal index): ue [nue], rptr [nue + 1], rlist [nrec]
  int64_t nue = 0;
  int64_t* d_ue = nullptr;
  int32_t* d_rptr = nullptr;
  int32_t* d_rlist = nullptr;
  // recorded run
  bool recorded = false;
  double dt = 0.0;
  int64_t nsteps = 0, every = 1;
  std::vector<int64_t> k_step;  // the solver's step counter at the start of each step (amplitude samples)
  std::vector<void*> ckpt;      // internal-layout states at steps 0, C, 2C, ...
  double* d_traces = nullptr;   // [nsteps][nrec]
  // gradient tables: pairs (alpha, alpha') of degree-N indices grouped by
  // gamma = alpha + alpha' (CSR over the degree-2N lattice), 1 / alpha!, and
  // G[gamma][beta] = C_b (gamma + beta)! / beta!
  int32_t* d_gptr = nullptr;
  uint32_t* d_pairs = nullptr;
  void* d_invf = nullptr;
  void* d_gw = nullptr;
  int ngam = 0;
  int32_t* d_split = nullptr;  // gamma ranges of the gradient kernel's warps [kGradWarps + 1]
  bool grad_ready = false;  // the gradient kernel's shared-memory attribute is set
  int nsm = 0;              // SMs of the device
  // adjoint state (internal layout [G][4][Np][V]): kap, rho, y; the recompute's
  // state ping-pong and residual; the pressure brackets of every stage of a
  // segment [5 C][G][Np][V]; the c^2 gradient [K][Mp] (internal element order)
  void* kap = nullptr;
  void* rho = nullptr;
  void* yi = nullptr;
  void* qa[2] = {nullptr, nullptr};
  void* rs = nullptr;
  void* brk = nullptr;
  size_t brk_bytes = 0;
  void* gc = nullptr;
  double* d_g = nullptr;  // [nsteps][nrec] trace cotangents
};

namespace {

__host__ __device__ inline size_t iidx(int64_t e, int i, int f, int Np, int V) {
  return ((size_t(e / V) * 4 + f) * Np + i) * V + size_t(e % V);
}

// traces: out[r] = sum_i B_r[i] p_{e_r}[i], one warp per receiver
template <typename real>
__global__ void sample_kernel(const real* __restrict__ q, int64_t nrec, const int64_t* __restrict__ el,
                              const real* __restrict__ vec, int Np, int V, double* __restrict__ out) {
  const int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (r >= nrec) return;  // warp-uniform
  double acc = 0.0;
  for (int i = lane; i < Np; i += 32) acc += double(vec[r * Np + i]) * double(q[iidx(el[r], i, 0, Np, V)]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[r] = acc;
}

// kap_p[e] += sum_{r at e} g[r] M^{-1} B_r: one block per receiving element,
// its receivers summed in order (rptr: CSR over the elements ue that hold
// receivers, rlist: receiver indices), threads over coefficients
template <typename real>
__global__ void receiver_adjoint_kernel(real* __restrict__ kap, const int64_t* __restrict__ ue,
                                        const int32_t* __restrict__ rptr, const int32_t* __restrict__ rlist,
                                        const real* __restrict__ dual, const double* __restrict__ g, int Np, int V) {
  const int u = blockIdx.x;
  for (int i = threadIdx.x; i < Np; i += blockDim.x) {
    real acc = 0;
    for (int x = rptr[u]; x < rptr[u + 1]; ++x) acc += real(g[rlist[x]]) * dual[size_t(rlist[x]) * Np + i];
    kap[iidx(ue[u], i, 0, Np, V)] += acc;
  }
}

// gc[e][b] += dt sum_gamma G[gamma][b] sum_{(a, a') in pairs(gamma)} rho_p[e][a] / a! * v[e][a'] / a'!.
// A block of kGradWarps warps takes 32 consecutive (internal) elements, one
// per lane. The operands are staged once per block as [Np][32] columns; warp
// q walks the gamma range [split.c[q], split.c[q + 1]) (ranges balanced by
// pair count on the host), all its lanes in step over the same pair list, so
// table words are broadcast loads and each lane reads only its own column
// (no bank conflicts, no imbalance between lanes); split [kGradWarps + 1]
// holds the ranges (device memory). The warps' partial sums
// are added in warp order (deterministic). rho_p is field 0 of the internal
// [G][4][Np][V] layout, v the pressure bracket [G][Np][V]. Pair words hold
// (32 a) | (32 a') << 16, the operand offsets in the columns. With SMEM the
// tables (G, pairs, row pointers; tab_bytes) are first copied into shared
// memory, otherwise read from global memory (uniform loads).
template <typename real, bool SMEM>
__global__ void __launch_bounds__(32 * kGradWarps) adj_grad_kernel(
    const real* __restrict__ rho, const real* __restrict__ v, real* __restrict__ gc, int64_t K, int Np, int Mp, int V,
    int ngam, const int32_t* __restrict__ gptr_g, const uint32_t* __restrict__ pairs_g, const real* __restrict__ invf,
    const real* __restrict__ gw_g, real dt, int tab_bytes, const int32_t* __restrict__ split) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int32_t* gptr = gptr_g;
  const uint32_t* pairs = pairs_g;
  const real* gw = gw_g;
  if constexpr (SMEM) {
    real* gws = reinterpret_cast<real*>(sm_raw);
    uint32_t* ps = reinterpret_cast<uint32_t*>(gws + size_t(ngam) * Mp);
    int32_t* gp = reinterpret_cast<int32_t*>(ps + size_t(Np) * Np);
    for (int x = threadIdx.x; x < ngam * Mp; x += blockDim.x) gws[x] = gw_g[x];
    for (int x = threadIdx.x; x < Np * Np; x += blockDim.x) ps[x] = pairs_g[x];
    for (int x = threadIdx.x; x <= ngam; x += blockDim.x) gp[x] = gptr_g[x];
    gptr = gp;
    pairs = ps;
    gw = gws;
  }
  real* rs0 = reinterpret_cast<real*>(sm_raw + tab_bytes);
  real* vs0 = rs0 + size_t(Np) * 32;
  real* part = vs0 + size_t(Np) * 32;  // [kGradWarps][Mp][32]
  const real* rs = rs0 + lane;
  const real* vs = vs0 + lane;
  const int c_lo = split[w], c_hi = split[w + 1];
  for (int64_t e0 = int64_t(blockIdx.x) * 32; e0 < K; e0 += int64_t(gridDim.x) * 32) {
    {  // stage the 32 elements' operands, warp w taking rows w, w + 8, ...
      const int64_t e = e0 + lane;
      const bool ok = e < K;
      const int64_t g = ok ? e / V : 0;
      const int l = ok ? int(e % V) : 0;
      for (int i = w; i < Np; i += kGradWarps) {
        const real f = invf[i];
        rs0[i * 32 + lane] = ok ? rho[(size_t(g) * 4 * Np + i) * V + l] * f : real(0);
        vs0[i * 32 + lane] = ok ? v[(size_t(g) * Np + i) * V + l] * f : real(0);
      }
    }
    __syncthreads();
    real acc[kMaxMp];
#pragma unroll
    for (int b = 0; b < kMaxMp; ++b) acc[b] = real(0);
    int p = gptr[c_lo];
    for (int c = c_lo; c < c_hi; ++c) {
      const int p1 = gptr[c + 1];
      real wg = 0;
#pragma unroll 4
      for (; p < p1; ++p) {
        const uint32_t ab = pairs[p];
        wg += rs[ab & 0xffffu] * vs[ab >> 16];
      }
#pragma unroll
      for (int b = 0; b < kMaxMp; ++b)
        if (b < Mp) acc[b] += wg * gw[size_t(c) * Mp + b];
    }
#pragma unroll
    for (int b = 0; b < kMaxMp; ++b)
      if (b < Mp) part[(size_t(w) * Mp + b) * 32 + lane] = acc[b];
    __syncthreads();
    for (int x = threadIdx.x; x < Mp * 32; x += blockDim.x) {
      const int b = x / 32, ln = x % 32;
      real sum = 0;
      for (int q = 0; q < kGradWarps; ++q) sum += part[(size_t(q) * Mp + b) * 32 + ln];
      if (e0 + ln < K) gc[size_t(e0 + ln) * Mp + b] += dt * sum;
    }
    __syncthreads();
  }
}

bbw_status dalloc(void** p, size_t bytes) {
  if (*p) return BBW_OK;
  BBW_CUDA(cudaMalloc(p, bytes));
  BBW_CUDA(cudaMemset(*p, 0, bytes));
  return BBW_OK;
}

template <typename real>
bbw_status upload_real(const std::vector<double>& h, void** d) {
  std::vector<real> r(h.begin(), h.end());
  bbw_status st = dalloc(d, r.size() * sizeof(real));
  if (st != BBW_OK) return st;
  BBW_CUDA(cudaMemcpy(*d, r.data(), r.size() * sizeof(real), cudaMemcpyHostToDevice));
  return BBW_OK;
}

// The gradient tables of the degree-2N product (see the file comment).
template <typename real>
bbw_status build_tables(bbw_solver* s, AdjointData* a) {
  if (a->d_gptr) return BBW_OK;
  const int N = s->N, M = s->M, Np = s->Np, Mp = s->Mp;
  const auto A = bbw::lattice(N);
  const auto B = bbw::lattice(M);
  const auto G2 = bbw::lattice(2 * N);
  auto f = [](int n) { return bbw::factorial(n); };
  auto idx2n = [&](const std::array<int, 4>& g) {  // position of gamma in the degree-2N library order
    return bbw::idx3(2 * N, g[1], g[2], g[3]);
  };
  const int ngam = int(G2.size());
  std::vector<std::vector<uint32_t>> by(static_cast<size_t>(ngam));
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      std::array<int, 4> g;
      for (int x = 0; x < 4; ++x) g[x] = A[size_t(i)][x] + A[size_t(j)][x];
      // offsets of the two operands in the warp's staged [Np][32] columns
      by[size_t(idx2n(g))].push_back(uint32_t(32 * i) | (uint32_t(32 * j) << 16));
    }
  std::vector<int32_t> gptr(size_t(ngam) + 1, 0);
  std::vector<uint32_t> pairs;
  for (int c = 0; c < ngam; ++c) {
    gptr[size_t(c)] = int32_t(pairs.size());
    pairs.insert(pairs.end(), by[size_t(c)].begin(), by[size_t(c)].end());
  }
  gptr[size_t(ngam)] = int32_t(pairs.size());
  // warp q takes the gammas whose cumulative cost (pairs + Mp weights) falls
  // in its q-th share
  {
    std::vector<double> cum(size_t(ngam) + 1, 0.0);
    for (int c = 0; c < ngam; ++c) cum[size_t(c) + 1] = cum[size_t(c)] + double(gptr[size_t(c) + 1] - gptr[size_t(c)] + Mp);
    std::vector<int32_t> split(size_t(kGradWarps) + 1, 0);
    int c = 0;
    for (int q = 1; q < kGradWarps; ++q) {
      const double target = cum[size_t(ngam)] * q / kGradWarps;
      while (c < ngam && cum[size_t(c)] < target) ++c;
      split[size_t(q)] = c;
    }
    split[size_t(kGradWarps)] = ngam;
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_split), split.size() * sizeof(int32_t)));
    BBW_CUDA(cudaMemcpy(a->d_split, split.data(), split.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  const double cb = 6.0 * f(N) * f(N) * f(M) / f(2 * N + M + 3);
  std::vector<double> gw(size_t(ngam) * Mp);
  std::vector<double> invf(static_cast<size_t>(Np));
  for (int c = 0; c < ngam; ++c)
    for (int b = 0; b < Mp; ++b) {
      double x = cb;
      for (int q = 0; q < 4; ++q) x *= f(G2[size_t(c)][q] + B[size_t(b)][q]) / f(B[size_t(b)][q]);
      gw[size_t(c) * Mp + b] = x;
    }
  for (int i = 0; i < Np; ++i) {
    const auto& ai = A[size_t(i)];
    invf[size_t(i)] = 1.0 / (f(ai[0]) * f(ai[1]) * f(ai[2]) * f(ai[3]));
  }
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_gptr), gptr.size() * sizeof(int32_t)));
  BBW_CUDA(cudaMemcpy(a->d_gptr, gptr.data(), gptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_pairs), pairs.size() * sizeof(uint32_t)));
  BBW_CUDA(cudaMemcpy(a->d_pairs, pairs.data(), pairs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  a->ngam = ngam;
  bbw_status st = upload_real<real>(gw, &a->d_gw);
  if (st == BBW_OK) st = upload_real<real>(invf, &a->d_invf);
  return st;
}

AdjointData* adj_of(bbw_solver* s) {
  if (!s->adj) s->adj = new AdjointData();
  return s->adj;
}

// Forget the recorded run. Buffers stay allocated for the next run unless
// release is set.
void free_run(AdjointData* a, bool release = false) {
  if (release) {
    for (void* p : a->ckpt)
      if (p) cudaFree(p);
    a->ckpt.clear();
    if (a->brk) cudaFree(a->brk);
    a->brk = nullptr;
    a->brk_bytes = 0;
  }
  if (a->d_traces) cudaFree(a->d_traces);
  a->d_traces = nullptr;
  a->recorded = false;
}

// The solver's launch parameters for a stage on explicit buffers.
template <typename real>
bbw::StageParams<real> stage_params(bbw_solver* s, const void* qin, void* qout, void* res) {
  bbw::StageParams<real> P;
  P.qin = static_cast<const real*>(qin);
  P.qout = static_cast<real*>(qout);
  P.res = static_cast<real*>(res);
  P.c2 = static_cast<const real*>(s->d_c2);
  P.geom = static_cast<const real*>(s->d_geom);
  P.conn = s->d_conn;
  P.tables = s->op->tables;
  P.G = s->G;
  P.a = real(0);
  P.b = real(0);
  P.dt = real(0);
  P.tau_p = real(s->tau_p);
  P.tau_u = real(s->tau_u);
  P.status = s->d_status;
  return P;
}

// One forward stage qin -> qout (res updated) of step `step`, storing its
// pressure bracket in vout.
template <typename real>
bbw_status forward_stage(bbw_solver* s, const void* qin, void* qout, void* res, int stage, double dt, int64_t step,
                         void* vout) {
  double ca[5], cb[5];
  bbw_lsrk_coeffs(ca, cb, nullptr);
  bbw::StageParams<real> P = stage_params<real>(s, qin, qout, res);
  P.a = real(ca[stage]);
  P.b = real(cb[stage]);
  P.dt = real(dt);
  bbw::set_stage_sources<bbw::StageParams<real>, real>(s, P, step, stage, true);
  P.vout = static_cast<real*>(vout);
  BBW_CUDA(s->ops->launch_stage(s->M, s->prec == 64, &P, s->grid_stage, s->stream));
  return BBW_OK;
}

// Adjoint of stage `stage` whose forward pressure bracket is vbr.
template <typename real>
bbw_status adjoint_stage(bbw_solver* s, AdjointData* a, const void* vbr, int stage, double dt) {
  double ca[5], cb[5];
  bbw_lsrk_coeffs(ca, cb, nullptr);
  cudaStream_t st = s->stream;
  // rho_t = a_{s+1} rho + b_s kap (rho holds rho_t of the stage after; at the
  // last stage of a step the incoming res cotangent is zero, a_0 = 0); y
  bbw::AdjPreParams<real> Q;
  Q.rho = static_cast<real*>(a->rho);
  Q.kap = static_cast<const real*>(a->kap);
  Q.c2 = static_cast<const real*>(s->d_c2);
  Q.geom = static_cast<const real*>(s->d_geom);
  Q.y = static_cast<real*>(a->yi);
  Q.tables = s->op->tables;
  Q.G = s->G;
  Q.a = stage == 4 ? real(0) : real(ca[stage + 1]);
  Q.b = real(cb[stage]);
  BBW_CUDA(s->ops->launch_adj_pre(s->M, s->prec == 64, &Q, s->grid_stage, st));
  // kap -= dt |D| A_{-tau}(y)
  bbw::StageParams<real> P = stage_params<real>(s, a->yi, a->kap, a->kap);
  P.tau_p = real(-s->tau_p);
  P.tau_u = real(-s->tau_u);
  P.dt = real(dt);
  P.accumulate = 1;
  bbw::set_stage_sources<bbw::StageParams<real>, real>(s, P, 0, stage, false);
  BBW_CUDA(s->ops->launch_spatial(s->M, s->prec == 64, &P, s->grid_stage, st));
  // gc += dt rho_t,p^T T_beta v
  const size_t ops = (size_t(2) * s->Np + size_t(kGradWarps) * s->Mp) * 32 * sizeof(real);  // staged operands, partials
  const size_t tab = (size_t(a->ngam) * s->Mp * sizeof(real) + size_t(s->Np) * s->Np * 4 + size_t(a->ngam + 1) * 4 +
                      15) / 16 * 16;
  const size_t cap = size_t(bbw::kSmemPerCta);
  const bool in_smem = tab + ops <= cap;
  const size_t bytes = (in_smem ? tab : 0) + ops;
  if (bytes > cap) return fail(BBW_ERR_ARG, "adjoint gradient: staged operands exceed shared memory");
  if (!a->grad_ready) {
    BBW_CUDA(cudaFuncSetAttribute(adj_grad_kernel<real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(cap)));
    BBW_CUDA(cudaFuncSetAttribute(adj_grad_kernel<real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(cap)));
    int dev = 0;
    BBW_CUDA(cudaGetDevice(&dev));
    BBW_CUDA(cudaDeviceGetAttribute(&a->nsm, cudaDevAttrMultiProcessorCount, dev));
    a->grad_ready = true;
  }
  // blocks per SM: as many as the shared memory holds (at most 8)
  const int per_sm = int(std::max<size_t>(1, std::min<size_t>(8, cap / bytes)));
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((s->K + 31) / 32, int64_t(std::max(a->nsm, 1)) * per_sm)));
  auto launch = [&](auto kern) {
    kern<<<blocks, 32 * kGradWarps, bytes, st>>>(
        static_cast<const real*>(a->rho), static_cast<const real*>(vbr), static_cast<real*>(a->gc), s->K, s->Np, s->Mp,
        s->V, a->ngam, a->d_gptr, a->d_pairs, static_cast<const real*>(a->d_invf), static_cast<const real*>(a->d_gw),
        real(dt), in_smem ? int(tab) : 0, a->d_split);
  };
  if (in_smem)
    launch(adj_grad_kernel<real, true>);
  else
    launch(adj_grad_kernel<real, false>);
  BBW_CUDA(cudaGetLastError());
  return BBW_OK;
}

template <typename real>
bbw_status record(bbw_solver* s, double dt, int64_t nsteps, int64_t every, double* traces) {
  AdjointData* a = adj_of(s);
  free_run(a);
  const size_t bytes = s->nstate_internal() * sizeof(real);
  const size_t pbytes = size_t(s->G) * s->V * s->Np * sizeof(real);  // one pressure field, internal layout
  a->dt = dt;
  a->nsteps = nsteps;
  a->every = every;
  a->k_step.assign(size_t(nsteps), 0);
  // every == 0: keep the pressure bracket of every stage of the run instead
  // of checkpoints (the adjoint then recomputes nothing); otherwise release
  // a bracket buffer larger than the adjoint's segments need
  const size_t need_brk = every == 0 ? size_t(nsteps) * 5 * pbytes : size_t(every) * 5 * pbytes;
  if (a->brk && (every == 0 ? a->brk_bytes < need_brk : a->brk_bytes > 2 * need_brk)) {
    cudaFree(a->brk);
    a->brk = nullptr;
    a->brk_bytes = 0;
  }
  if (every == 0 && !a->brk) {
    size_t free_b = 0, total_b = 0;
    BBW_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (need_brk > free_b)
      return fail(BBW_ERR_ARG, "keeping every stage's pressure bracket needs " + std::to_string(need_brk >> 20) +
                                   " MiB of device memory, " + std::to_string(free_b >> 20) +
                                   " MiB are free: use checkpoint_every >= 1");
    BBW_CUDA(cudaMalloc(&a->brk, need_brk));
    a->brk_bytes = need_brk;
  }
  const int64_t nck = every == 0 ? 0 : std::max<int64_t>((nsteps + every - 1) / every, 1);
  while (int64_t(a->ckpt.size()) > nck) {  // keep the buffers of earlier runs, drop extras
    if (a->ckpt.back()) cudaFree(a->ckpt.back());
    a->ckpt.pop_back();
  }
  a->ckpt.resize(size_t(nck), nullptr);
  for (auto& c : a->ckpt) {
    bbw_status st = dalloc(&c, bytes);
    if (st != BBW_OK) return st;
  }
  if (a->nrec > 0) BBW_CUDA(cudaMalloc(&a->d_traces, size_t(nsteps) * a->nrec * sizeof(double)));
  const int threads = 128;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (every > 0 && n % every == 0)
      BBW_CUDA(cudaMemcpyAsync(a->ckpt[size_t(n / every)], s->q[s->cur], bytes, cudaMemcpyDeviceToDevice, s->stream));
    a->k_step[size_t(n)] = s->steps;
    bbw_status st = BBW_OK;
    if (every == 0) {
      for (int sg = 0; sg < 5 && st == BBW_OK; ++sg) {
        s->vout = static_cast<char*>(a->brk) + size_t(n * 5 + sg) * pbytes;
        st = bbw_stage(s, sg, dt);
      }
      s->vout = nullptr;
    } else {
      st = bbw_step(s, dt, 1);
    }
    if (st != BBW_OK) return st;
    if (a->nrec > 0)
      sample_kernel<real><<<int((a->nrec * 32 + threads - 1) / threads), threads, 0, s->stream>>>(
          static_cast<const real*>(s->q[s->cur]), a->nrec, a->d_rec_elem, static_cast<const real*>(a->d_rec_vec),
          s->Np, s->V, a->d_traces + size_t(n) * a->nrec);
  }
  BBW_CUDA(cudaGetLastError());
  if (traces && a->nrec > 0)
    BBW_CUDA(cudaMemcpyAsync(traces, a->d_traces, size_t(nsteps) * a->nrec * sizeof(double), cudaMemcpyDeviceToHost,
                             s->stream));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  a->recorded = true;
  return bbw::check_status(s);
}

template <typename real>
bbw_status adjoint(bbw_solver* s, const double* g, double* grad_c2, double* grad_q0) {
  AdjointData* a = s->adj;
  if (!a || !a->recorded) return fail(BBW_ERR_ARG, "no recorded run (call bbw_record first)");
  bbw_status st = build_tables<real>(s, a);
  if (st != BBW_OK) return st;
  const int64_t K = s->K;
  const int Np = s->Np, Mp = s->Mp;
  const size_t bytes = s->nstate_internal() * sizeof(real);
  const size_t pbytes = size_t(s->G) * s->V * Np * sizeof(real);  // one pressure field, internal layout
  for (void** b : {&a->kap, &a->rho, &a->yi, &a->qa[0], &a->qa[1], &a->rs}) {
    st = dalloc(b, bytes);
    if (st != BBW_OK) return st;
  }
  st = dalloc(&a->gc, size_t(K) * Mp * sizeof(real));
  if (st != BBW_OK) return st;
  const size_t need = size_t(a->every) * 5 * pbytes;  // 0 when the recorded run kept every bracket
  if (a->brk_bytes < need) {
    if (a->brk) cudaFree(a->brk);
    a->brk = nullptr;
    a->brk_bytes = 0;
    BBW_CUDA(cudaMalloc(&a->brk, need));
    a->brk_bytes = need;
  }
  if (a->d_g) cudaFree(a->d_g);
  a->d_g = nullptr;
  if (a->nrec > 0 && g) {
    const size_t ng = size_t(a->nsteps) * a->nrec;
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_g), ng * sizeof(double)));
    BBW_CUDA(cudaMemcpy(a->d_g, g, ng * sizeof(double), cudaMemcpyHostToDevice));
  }
  cudaStream_t sm = s->stream;
  BBW_CUDA(cudaMemsetAsync(a->kap, 0, bytes, sm));
  BBW_CUDA(cudaMemsetAsync(a->rho, 0, bytes, sm));
  BBW_CUDA(cudaMemsetAsync(a->gc, 0, size_t(K) * Mp * sizeof(real), sm));
  auto bracket = [&](int64_t i) { return static_cast<void*>(static_cast<char*>(a->brk) + size_t(i) * pbytes); };
  const double dt = a->dt;
  const bool kept = a->every == 0;  // the recorded run kept every bracket: one segment, nothing recomputed
  const int64_t nseg = kept ? 1 : int64_t(a->ckpt.size());
  for (int64_t k = nseg - 1; k >= 0; --k) {
    const int64_t n0 = kept ? 0 : k * a->every, n1 = kept ? a->nsteps : std::min(a->nsteps, n0 + a->every);
    if (!kept) {
      // recompute the segment from its checkpoint, keeping every stage's bracket
      BBW_CUDA(cudaMemcpyAsync(a->qa[0], a->ckpt[size_t(k)], bytes, cudaMemcpyDeviceToDevice, sm));
      int cur = 0;
      for (int64_t n = n0; n < n1; ++n)
        for (int sg = 0; sg < 5; ++sg) {
          st = forward_stage<real>(s, a->qa[cur], a->qa[1 - cur], a->rs, sg, dt, a->k_step[size_t(n)],
                                   bracket((n - n0) * 5 + sg));
          if (st != BBW_OK) return st;
          cur = 1 - cur;
        }
    }
    for (int64_t n = n1 - 1; n >= n0; --n) {
      // cotangent of the traces after step n
      if (a->d_g) {
        receiver_adjoint_kernel<real><<<int(a->nue), 64, 0, sm>>>(
            static_cast<real*>(a->kap), a->d_ue, a->d_rptr, a->d_rlist, static_cast<const real*>(a->d_rec_dual),
            a->d_g + size_t(n) * a->nrec, Np, s->V);
        BBW_CUDA(cudaGetLastError());
      }
      for (int sg = 4; sg >= 0; --sg) {
        st = adjoint_stage<real>(s, a, bracket((n - n0) * 5 + sg), sg, dt);
        if (st != BBW_OK) return st;
      }
      // the step's res enters only through stage 0 (a_0 = 0): the res
      // cotangent is zero at every step boundary (a_next = 0 at stage 4)
    }
  }
  BBW_CUDA(cudaStreamSynchronize(sm));
  st = bbw::check_status(s);
  if (st != BBW_OK) return st;
  // back to the caller's element order
  if (grad_c2) {
    std::vector<real> h(size_t(K) * Mp);
    BBW_CUDA(cudaMemcpy(h.data(), a->gc, h.size() * sizeof(real), cudaMemcpyDeviceToHost));
    for (int64_t e = 0; e < K; ++e)
      for (int b = 0; b < Mp; ++b) grad_c2[size_t(s->user(e)) * Mp + b] = double(h[size_t(e) * Mp + b]);
  }
  if (grad_q0) {
    // qbar = M kap per element and field (the reference mass, in FP64 on the host)
    const size_t nf = size_t(K) * Np;
    std::vector<double> kh(4 * nf);
    void* tmp = nullptr;
    BBW_CUDA(cudaMalloc(&tmp, 4 * nf * sizeof(double)));
    cudaError_t e1 = bbw::copy_to_user(a->kap, s->prec, tmp, 64, K, Np, s->V, s->d_inv, sm);
    if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(kh.data(), tmp, 4 * nf * sizeof(double), cudaMemcpyDeviceToHost, sm);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(sm);
    cudaFree(tmp);
    if (e1 != cudaSuccess) return fail(BBW_ERR_CUDA, std::string("state gradient download: ") + cudaGetErrorString(e1));
    const auto A = bbw::lattice(s->N);
    auto f = [](int n) { return bbw::factorial(n); };
    std::vector<double> mass(size_t(Np) * Np);
    for (int i = 0; i < Np; ++i)
      for (int j = 0; j < Np; ++j) {
        double m = 6.0 / f(2 * s->N + 3) * f(s->N) * f(s->N);
        for (int x = 0; x < 4; ++x)
          m *= f(A[size_t(i)][x] + A[size_t(j)][x]) / (f(A[size_t(i)][x]) * f(A[size_t(j)][x]));
        mass[size_t(i) * Np + j] = m;
      }
    for (size_t r = 0; r < 4 * size_t(K); ++r) {
      const double* x = kh.data() + r * Np;
      double* y = grad_q0 + r * Np;
      for (int i = 0; i < Np; ++i) {
        double acc = 0.0;
        for (int j = 0; j < Np; ++j) acc += mass[size_t(i) * Np + j] * x[j];
        y[i] = acc;
      }
    }
  }
  return BBW_OK;
}

}  // namespace

namespace bbw {

void free_adjoint(bbw_solver* s) {
  AdjointData* a = s->adj;
  if (!a) return;
  free_run(a, true);
  for (void* p : {static_cast<void*>(a->d_rec_elem), a->d_rec_vec, a->d_rec_dual, static_cast<void*>(a->d_ue),
                  static_cast<void*>(a->d_rptr), static_cast<void*>(a->d_rlist), static_cast<void*>(a->d_gptr),
                  static_cast<void*>(a->d_pairs), static_cast<void*>(a->d_split), a->d_invf, a->d_gw, a->kap, a->rho, a->yi, a->qa[0], a->qa[1],
                  a->rs, a->gc, static_cast<void*>(a->d_g)})
    if (p) cudaFree(p);
  delete a;
  s->adj = nullptr;
}

}  // namespace bbw

extern "C" {

bbw_status bbw_set_receivers(bbw_solver* s, int64_t nrec, const double* xyz, int64_t* elems) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (nrec < 0 || (nrec > 0 && !xyz)) return fail(BBW_ERR_ARG, "bad receiver list");
  AdjointData* a = adj_of(s);
  std::vector<int64_t> el(static_cast<size_t>(nrec), 0);
  std::vector<double> vec(static_cast<size_t>(nrec) * s->Np, 0.0), dual(vec.size(), 0.0);
  const auto A = bbw::lattice(s->N);
  for (int64_t r = 0; r < nrec; ++r) {
    // locate (lowest element index on shared faces) and evaluate the basis
    const double* x = xyz + 3 * r;
    int64_t found = -1;
    double lam[4] = {0, 0, 0, 0};
    for (int64_t e = 0; e < s->K && found < 0; ++e) {
      const double* gr = &s->grad[size_t(e) * 12];
      const double* v0 = &s->vxyz[size_t(s->etov[size_t(e) * 4]) * 3];
      double l[4];
      bool inside = true;
      for (int m = 0; m < 4; ++m) {
        l[m] = (m == 0 ? 1.0 : 0.0);
        for (int d = 0; d < 3; ++d) l[m] += gr[3 * m + d] * (x[d] - v0[d]);
        inside = inside && l[m] >= -1e-12;
      }
      if (inside) {
        found = e;
        std::memcpy(lam, l, sizeof(lam));
      }
    }
    if (found < 0) return fail(BBW_ERR_ARG, "receiver " + std::to_string(r) + " lies outside the mesh");
    el[size_t(r)] = found;
    std::vector<double> b(size_t(s->Np));
    for (size_t i = 0; i < A.size(); ++i) {
      double v = bbw::factorial(s->N) /
                 (bbw::factorial(A[i][0]) * bbw::factorial(A[i][1]) * bbw::factorial(A[i][2]) * bbw::factorial(A[i][3]));
      for (int m = 0; m < 4; ++m) v *= std::pow(std::max(lam[m], 0.0), A[i][m]);
      vec[size_t(r) * s->Np + i] = v;
      b[i] = v;
    }
    if (!bbw::solve_mass(s->N, b)) return fail(BBW_ERR_ARG, "mass matrix factorisation failed");
    std::copy(b.begin(), b.end(), dual.begin() + ptrdiff_t(size_t(r) * s->Np));
  }
  for (void** p : {reinterpret_cast<void**>(&a->d_rec_elem), &a->d_rec_vec, &a->d_rec_dual,
                   reinterpret_cast<void**>(&a->d_ue), reinterpret_cast<void**>(&a->d_rptr),
                   reinterpret_cast<void**>(&a->d_rlist)}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  a->nue = 0;
  a->nrec = nrec;
  a->rec_elem = el;
  free_run(a);
  if (nrec > 0) {
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_rec_elem), size_t(nrec) * sizeof(int64_t)));
    std::vector<int64_t> slots(el.size());
    for (size_t r = 0; r < el.size(); ++r) slots[r] = s->slot(el[r]);  // internal element order
    BBW_CUDA(cudaMemcpy(a->d_rec_elem, slots.data(), size_t(nrec) * sizeof(int64_t), cudaMemcpyHostToDevice));
    // receivers grouped by element, each group in receiver order
    std::vector<int32_t> order(slots.size());
    for (size_t r = 0; r < order.size(); ++r) order[r] = int32_t(r);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return slots[size_t(x)] < slots[size_t(y)]; });
    std::vector<int64_t> ue;
    std::vector<int32_t> rptr;
    for (size_t x = 0; x < order.size(); ++x) {
      if (x == 0 || slots[size_t(order[x])] != slots[size_t(order[x - 1])]) {
        ue.push_back(slots[size_t(order[x])]);
        rptr.push_back(int32_t(x));
      }
    }
    rptr.push_back(int32_t(order.size()));
    a->nue = int64_t(ue.size());
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_ue), ue.size() * sizeof(int64_t)));
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_rptr), rptr.size() * sizeof(int32_t)));
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_rlist), order.size() * sizeof(int32_t)));
    BBW_CUDA(cudaMemcpy(a->d_ue, ue.data(), ue.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    BBW_CUDA(cudaMemcpy(a->d_rptr, rptr.data(), rptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    BBW_CUDA(cudaMemcpy(a->d_rlist, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    bbw_status st = s->prec == 64 ? upload_real<double>(vec, &a->d_rec_vec) : upload_real<float>(vec, &a->d_rec_vec);
    if (st == BBW_OK)
      st = s->prec == 64 ? upload_real<double>(dual, &a->d_rec_dual) : upload_real<float>(dual, &a->d_rec_dual);
    if (st != BBW_OK) return st;
  }
  if (elems) std::copy(el.begin(), el.end(), elems);
  return BBW_OK;
}

bbw_status bbw_record(bbw_solver* s, double dt, int64_t nsteps, int64_t checkpoint_every, double* traces) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (nsteps < 1 || checkpoint_every < 0)
    return fail(BBW_ERR_ARG, "nsteps must be >= 1 and checkpoint_every >= 0");
  if (!std::isfinite(dt)) return fail(BBW_ERR_ARG, "dt is not finite");
  return s->prec == 64 ? record<double>(s, dt, nsteps, checkpoint_every, traces)
                       : record<float>(s, dt, nsteps, checkpoint_every, traces);
}

bbw_status bbw_adjoint(bbw_solver* s, const double* trace_grad, double* grad_c2, double* grad_q0) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return s->prec == 64 ? adjoint<double>(s, trace_grad, grad_c2, grad_q0)
                       : adjoint<float>(s, trace_grad, grad_c2, grad_q0);
}

}  // extern "C"
