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
//     L(tau)^T r = -M_w L(-tau) M_w^{-1} r
//                = -|D| M A_{-tau}( [ |D|^{-1} P~(c^2 . M^{-1} r_p) ; |D|^{-1} M^{-1} r_u ] ),
//
// A_{-tau} being the stage kernel's spatial operator (volume terms plus lifted
// fluxes, before the weight-adjusted update) with negated penalties. The
// adjoint stage therefore reuses the forward spatial kernel; only the
// element-local mass products are added here.
//
// Adjoint of one LSRK stage s (res' = a_s res + dt (L q + s), q' = q + b_s res'),
// from the cotangents (qb, rb) of (q', res'):
//     rt = rb + b_s qb;   qb += dt L^T rt;   rb = a_s rt
// (rb = a_s rt is folded into the next adjoint stage's rt = a_s rt + b_{s-1} qb);
//     gc2[k][beta] += dt (M^{-1} rt_p)_k^T T_beta v_k,
// with T_beta the mass matrix weighted by the degree-M Bernstein polynomial
// beta and v = (A_tau q + source) the pressure bracket of the forward stage.
//
// A recorded run keeps the state every C steps (checkpoints) and the start
// time of every step; the backward pass recomputes one checkpoint segment at
// a time, keeping the five stage inputs of each of its steps (memory: the
// checkpoints plus 5 C states).
//
// The element-local mass products are plain dense matrix products over all
// elements at once ([N_p x N_p] times [N_p x 4K], and the M_p weighted masses
// as one strided batch), done by cuBLAS in the solver's precision (no
// reduced-precision tensor-op modes).
#include <cublas_v2.h>
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

struct AdjointData {
  // receivers: element and Bernstein basis values B_i(lambda(x_r)) [nrec][Np]
  int64_t nrec = 0;
  std::vector<int64_t> rec_elem;
  int64_t* d_rec_elem = nullptr;
  void* d_rec_vec = nullptr;
  // recorded run
  bool recorded = false;
  double dt = 0.0;
  int64_t nsteps = 0, every = 1;
  std::vector<int64_t> k_step;  // the solver's step counter at the start of each step (amplitude samples)
  std::vector<void*> ckpt;      // internal-layout states at steps 0, C, 2C, ...
  double* d_traces = nullptr;   // [nsteps][nrec]
  // operator tables (real): M^{-1}, M [Np][Np]; T [Mp][Np][Np]
  void* d_minv = nullptr;
  void* d_mass = nullptr;
  void* d_tw = nullptr;
  void* d_vol = nullptr;    // [K] element volumes
  void* d_ivol = nullptr;   // [K] 1 / volume
  void* d_c2u = nullptr;    // [K][Mp] c^2 (for the WADG kernel)
  // work buffers in the ABI's field-major layout but the solver's internal
  // element order: [4][K][Np] (qb, rb, y, z, v), [K][Np] (yt), [K][Mp] (gc)
  void* qb = nullptr;
  void* rb = nullptr;
  void* y = nullptr;
  void* z = nullptr;
  void* v = nullptr;
  void* yt = nullptr;
  void* gc = nullptr;
  // internal layout: spatial-kernel input/output, stage inputs, segment states, res
  void* yi = nullptr;
  void* zi = nullptr;
  void* qs[5] = {};
  void* rs = nullptr;
  std::vector<void*> seg;
  double* d_g = nullptr;  // [nsteps][nrec] trace cotangents
  void* u = nullptr;      // [Mp][K][Np] weighted-mass products T_beta v_p
  cublasHandle_t blas = nullptr;
};

namespace {

__host__ __device__ inline size_t iidx(int64_t e, int i, int f, int Np, int V) {
  return ((size_t(e / V) * 4 + f) * Np + i) * V + size_t(e % V);
}

// traces: out[r] = sum_i B_r[i] p_{e_r}[i]
template <typename real>
__global__ void sample_kernel(const real* __restrict__ q, int64_t nrec, const int64_t* __restrict__ el,
                              const real* __restrict__ vec, int Np, int V, double* __restrict__ out) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r >= nrec) return;
  double acc = 0.0;
  for (int i = 0; i < Np; ++i) acc += double(vec[r * Np + i]) * double(q[iidx(el[r], i, 0, Np, V)]);
  out[r] = acc;
}

// qb_p[e_r] += g[r] B_r, receivers in order (threads over coefficients)
template <typename real>
__global__ void receiver_adjoint_kernel(real* __restrict__ qb, int64_t K, int64_t nrec, const int64_t* __restrict__ el,
                                        const real* __restrict__ vec, const double* __restrict__ g, int Np) {
  for (int i = threadIdx.x; i < Np; i += blockDim.x)
    for (int64_t r = 0; r < nrec; ++r) qb[el[r] * Np + i] += real(g[r]) * vec[r * Np + i];
}

// x = a x + b y (elementwise)
template <typename real>
__global__ void axpby_kernel(real* __restrict__ x, const real* __restrict__ y, real a, real b, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    x[i] = a * x[i] + (y ? b * y[i] : real(0));
}

// user [nf][K][Np] -> internal [G][4][Np][V] (fields >= nf and padding zero),
// times scale[e] if given
template <typename real>
__global__ void to_internal_scaled(const real* __restrict__ in, real* __restrict__ out, int64_t K, int Np, int V,
                                   const real* __restrict__ scale, size_t n_internal) {
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n_internal; x += size_t(gridDim.x) * blockDim.x) {
    const int v = int(x % V);
    const size_t r = x / V;
    const int i = int(r % Np);
    const size_t r2 = r / Np;
    const int f = int(r2 % 4);
    const int64_t e = int64_t(r2 / 4) * V + v;
    out[x] = e < K ? in[(size_t(f) * K + e) * Np + i] * (scale ? scale[e] : real(1)) : real(0);
  }
}

// internal -> user, fields 0..nf-1, times scale[e] if given
template <typename real>
__global__ void to_user_scaled(const real* __restrict__ in, real* __restrict__ out, int64_t K, int Np, int V, int nf,
                               const real* __restrict__ scale) {
  const size_t n = size_t(nf) * K * Np;
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n; x += size_t(gridDim.x) * blockDim.x) {
    const int i = int(x % Np);
    const size_t r = x / Np;
    const int64_t e = int64_t(r % K);
    const int f = int(r / K);
    out[x] = in[iidx(e, i, f, Np, V)] * (scale ? scale[e] : real(1));
  }
}

// gc[e][b] += alpha sum_i yt[e][i] u[b][e][i]   (u_b = T_b v_p)
template <typename real>
__global__ void grad_c2_kernel(const real* __restrict__ u, const real* __restrict__ yt, real* __restrict__ gc,
                               int64_t K, int Mp, int Np, real alpha) {
  const size_t n = size_t(K) * Mp;
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n; x += size_t(gridDim.x) * blockDim.x) {
    const int b = int(x % Mp);
    const int64_t e = int64_t(x / Mp);
    const real* ub = u + (size_t(b) * K + e) * Np;
    const real* ye = yt + size_t(e) * Np;
    real acc = 0;
    for (int i = 0; i < Np; ++i) acc += ye[i] * ub[i];
    gc[x] += alpha * acc;
  }
}

// Y = alpha A X + beta Y for row-major A [Np][Np] and ncols element rows of
// Np values (X, Y: [ncols][Np], i.e. column-major Np x ncols).
cublasStatus_t gemm(cublasHandle_t h, const float* A, int Np, const float* X, float* Y, int64_t ncols, float alpha,
                    float beta) {
  return cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, Np, int(ncols), Np, &alpha, A, Np, X, Np, &beta, Y, Np);
}
cublasStatus_t gemm(cublasHandle_t h, const double* A, int Np, const double* X, double* Y, int64_t ncols,
                    double alpha, double beta) {
  return cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, Np, int(ncols), Np, &alpha, A, Np, X, Np, &beta, Y, Np);
}
// U_b = T_b X for b < Mp (T: [Mp][Np][Np] row-major; U: [Mp][ncols][Np])
cublasStatus_t gemm_batch(cublasHandle_t h, const float* T, int Np, const float* X, float* U, int64_t ncols, int Mp) {
  const float one = 1.f, zero = 0.f;
  return cublasSgemmStridedBatched(h, CUBLAS_OP_T, CUBLAS_OP_N, Np, int(ncols), Np, &one, T, Np,
                                   static_cast<long long>(Np) * Np, X, Np, 0, &zero, U, Np, static_cast<long long>(Np) * ncols, Mp);
}
cublasStatus_t gemm_batch(cublasHandle_t h, const double* T, int Np, const double* X, double* U, int64_t ncols,
                          int Mp) {
  const double one = 1.0, zero = 0.0;
  return cublasDgemmStridedBatched(h, CUBLAS_OP_T, CUBLAS_OP_N, Np, int(ncols), Np, &one, T, Np,
                                   static_cast<long long>(Np) * Np, X, Np, 0, &zero, U, Np, static_cast<long long>(Np) * ncols, Mp);
}

#define BBW_BLAS(call)                                                                        \
  do {                                                                                        \
    const cublasStatus_t b_ = (call);                                                         \
    if (b_ != CUBLAS_STATUS_SUCCESS)                                                          \
      return fail(BBW_ERR_CUDA, std::string(#call) + ": cuBLAS status " + std::to_string(int(b_))); \
  } while (0)

int blocks_for(size_t n) { return int(std::min<size_t>((n + 255) / 256, 152 * 32)); }

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

// mass, inverse mass and weighted masses of the reference element (volume 1)
template <typename real>
bbw_status build_tables(bbw_solver* s, AdjointData* a) {
  if (a->d_minv) return BBW_OK;
  const int N = s->N, M = s->M, Np = s->Np, Mp = s->Mp;
  const auto A = bbw::lattice(N);
  const auto B = bbw::lattice(M);
  auto mult = [&](int n, const std::array<int, 4>& x) {
    return bbw::factorial(n) / (bbw::factorial(x[0]) * bbw::factorial(x[1]) * bbw::factorial(x[2]) *
                                bbw::factorial(x[3]));
  };
  std::vector<double> mass(size_t(Np) * Np), minv(size_t(Np) * Np), tw(size_t(Mp) * Np * Np);
  // Dirichlet integral over the unit-volume reference element:
  // int lambda^g = 3! g! / (|g| + 3)!
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double m = 6.0 / bbw::factorial(2 * N + 3);
      for (int x = 0; x < 4; ++x) m *= bbw::factorial(A[i][x] + A[j][x]);
      mass[size_t(i) * Np + j] = mult(N, A[i]) * mult(N, A[j]) * m;
      for (int b = 0; b < Mp; ++b) {
        double w = 6.0 / bbw::factorial(2 * N + M + 3);
        for (int x = 0; x < 4; ++x) w *= bbw::factorial(A[i][x] + A[j][x] + B[b][x]);
        tw[(size_t(b) * Np + i) * Np + j] = mult(M, B[b]) * mult(N, A[i]) * mult(N, A[j]) * w;
      }
    }
  for (int j = 0; j < Np; ++j) {
    std::vector<double> col(size_t(Np), 0.0);
    col[size_t(j)] = 1.0;
    if (!bbw::solve_mass(N, col)) return fail(BBW_ERR_ARG, "mass matrix factorisation failed");
    for (int i = 0; i < Np; ++i) minv[size_t(i) * Np + j] = col[size_t(i)];
  }
  // element arrays in the solver's internal element order
  std::vector<double> vol(s->vol.size()), ivol(s->vol.size());
  for (size_t e = 0; e < vol.size(); ++e) {
    vol[e] = s->vol[size_t(s->user(int64_t(e)))];
    ivol[e] = 1.0 / vol[e];
  }
  bbw_status st = upload_real<real>(mass, &a->d_mass);
  if (st == BBW_OK) st = upload_real<real>(minv, &a->d_minv);
  if (st == BBW_OK) st = upload_real<real>(tw, &a->d_tw);
  if (st == BBW_OK) st = upload_real<real>(vol, &a->d_vol);
  if (st == BBW_OK) st = upload_real<real>(ivol, &a->d_ivol);
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
    for (void* p : a->seg)
      if (p) cudaFree(p);
    a->seg.clear();
  }
  if (a->d_traces) cudaFree(a->d_traces);
  a->d_traces = nullptr;
  a->recorded = false;
}

// One forward stage on explicit buffers: qin -> qout, res updated, time t.
template <typename real>
bbw_status forward_stage(bbw_solver* s, const void* qin, void* qout, void* res, int stage, double dt,
                         int64_t step) {
  double ca[5], cb[5];
  bbw_lsrk_coeffs(ca, cb, nullptr);
  bbw::StageParams<real> P;
  P.qin = static_cast<const real*>(qin);
  P.qout = static_cast<real*>(qout);
  P.res = static_cast<real*>(res);
  P.c2 = static_cast<const real*>(s->d_c2);
  P.geom = static_cast<const real*>(s->d_geom);
  P.conn = s->d_conn;
  P.tables = s->op->tables;
  P.G = s->G;
  P.a = real(ca[stage]);
  P.b = real(cb[stage]);
  P.dt = real(dt);
  P.tau_p = real(s->tau_p);
  P.tau_u = real(s->tau_u);
  bbw::set_stage_sources<bbw::StageParams<real>, real>(s, P, step, stage, true);
  P.status = s->d_status;
  BBW_CUDA(s->ops->launch_stage(s->M, s->prec == 64, &P, s->grid_stage, s->stream));
  return BBW_OK;
}

// Spatial operator alone: out = [bracket_p (+ sources at t + c_s dt), rhs_u]
// of qin (internal layout), penalties sgn * tau.
template <typename real>
bbw_status spatial(bbw_solver* s, const void* qin, void* out, double sgn, bool sources, int stage, int64_t step) {
  bbw::StageParams<real> P;
  P.qin = static_cast<const real*>(qin);
  P.qout = static_cast<real*>(out);
  P.res = static_cast<real*>(out);
  P.c2 = static_cast<const real*>(s->d_c2);
  P.geom = static_cast<const real*>(s->d_geom);
  P.conn = s->d_conn;
  P.tables = s->op->tables;
  P.G = s->G;
  P.a = real(0);
  P.b = real(0);
  P.dt = real(0);
  P.tau_p = real(sgn * s->tau_p);
  P.tau_u = real(sgn * s->tau_u);
  bbw::set_stage_sources<bbw::StageParams<real>, real>(s, P, step, stage, sources);
  P.status = s->d_status;
  BBW_CUDA(s->ops->launch_spatial(s->M, s->prec == 64, &P, s->grid_stage, s->stream));
  return BBW_OK;
}

template <typename real>
bbw_status wadg_user(bbw_solver* s, const void* in, const void* c2u, void* out) {
  bbw::WadgParams<real> P;
  P.rhs = static_cast<const real*>(in);
  P.c2 = static_cast<const real*>(c2u);
  P.out = static_cast<real*>(out);
  P.tables = s->op->tables;
  P.K = s->K;
  int team = 0, V = 1, gpc = 1;
  s->ops->launch_shape(s->M, s->prec == 64, &team, &V, &gpc);
  const int64_t tiles = (s->K + int64_t(V) * gpc - 1) / (int64_t(V) * gpc);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = int(std::min<int64_t>(tiles, int64_t(std::max(1, s->op->per_sm_wadg)) * std::max(1, nsm)));
  BBW_CUDA(s->ops->launch_wadg(s->M, s->prec == 64, &P, std::max(1, grid), s->stream));
  return BBW_OK;
}

// Adjoint of stage `stage` of the step starting at time t, whose stage input
// (internal layout) is qin; updates qb, rb (user layout) and gc.
template <typename real>
bbw_status adjoint_stage(bbw_solver* s, AdjointData* a, const void* qin, int stage, double dt, int64_t step) {
  double ca[5], cb[5], cc[5];
  bbw_lsrk_coeffs(ca, cb, cc);
  const int64_t K = s->K;
  const int Np = s->Np, Mp = s->Mp, V = s->V;
  const size_t nf = size_t(K) * Np;
  const int p = s->prec;
  real* qb = static_cast<real*>(a->qb);
  real* rb = static_cast<real*>(a->rb);
  real* y = static_cast<real*>(a->y);
  real* z = static_cast<real*>(a->z);
  real* v = static_cast<real*>(a->v);
  real* yt = static_cast<real*>(a->yt);
  const real* minv = static_cast<const real*>(a->d_minv);
  const real* mass = static_cast<const real*>(a->d_mass);
  const real* vol = static_cast<const real*>(a->d_vol);
  const real* ivol = static_cast<const real*>(a->d_ivol);
  cudaStream_t st = s->stream;
  // rt = a_{s+1} rt + b_s qb in rb (rb holds rt of the stage after; at the
  // last stage of a step the incoming res cotangent is zero, a_0 = 0)
  const real a_next = stage == 4 ? real(0) : real(ca[stage + 1]);
  axpby_kernel<real><<<blocks_for(4 * nf), 256, 0, st>>>(rb, qb, a_next, real(cb[stage]), 4 * nf);
  // yt = M^{-1} rt_p; y = [P~(c2 . yt); M^{-1} rt_u], scaled by 1/|D| into the grouped layout
  BBW_BLAS(gemm(a->blas, minv, Np, rb, yt, K, real(1), real(0)));
  bbw_status r = wadg_user<real>(s, yt, a->d_c2u, y);
  if (r != BBW_OK) return r;
  BBW_BLAS(gemm(a->blas, minv, Np, rb + nf, y + nf, 3 * K, real(1), real(0)));
  const size_t ni = s->nstate_internal();
  to_internal_scaled<real><<<blocks_for(ni), 256, 0, st>>>(y, static_cast<real*>(a->yi), K, Np, V, ivol, ni);
  BBW_CUDA(cudaGetLastError());
  // z = |D| A_{-tau}(y); v_p = (A_tau(q_s) + sources)_p
  r = spatial<real>(s, a->yi, a->zi, -1.0, false, stage, step);
  if (r != BBW_OK) return r;
  to_user_scaled<real><<<blocks_for(4 * nf), 256, 0, st>>>(static_cast<const real*>(a->zi), z, K, Np, V, 4, vol);
  r = spatial<real>(s, qin, a->zi, 1.0, true, stage, step);
  if (r != BBW_OK) return r;
  to_user_scaled<real><<<blocks_for(nf), 256, 0, st>>>(static_cast<const real*>(a->zi), v, K, Np, V, 1, nullptr);
  BBW_CUDA(cudaGetLastError());
  // qb -= dt M z; gc += dt yt^T T_b v_p
  BBW_BLAS(gemm(a->blas, mass, Np, z, qb, 4 * K, real(-dt), real(1)));
  BBW_BLAS(gemm_batch(a->blas, static_cast<const real*>(a->d_tw), Np, v, static_cast<real*>(a->u), K, Mp));
  grad_c2_kernel<real><<<blocks_for(size_t(K) * Mp), 256, 0, st>>>(static_cast<const real*>(a->u), yt,
                                                                     static_cast<real*>(a->gc), K, Mp, Np, real(dt));
  BBW_CUDA(cudaGetLastError());
  return BBW_OK;
}

template <typename real>
bbw_status record(bbw_solver* s, double dt, int64_t nsteps, int64_t every, double* traces) {
  AdjointData* a = adj_of(s);
  free_run(a);
  const size_t bytes = s->nstate_internal() * sizeof(real);
  a->dt = dt;
  a->nsteps = nsteps;
  a->every = every;
  a->k_step.assign(size_t(nsteps), 0);
  const int64_t nck = std::max<int64_t>((nsteps + every - 1) / every, 1);
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
    if (n % every == 0)
      BBW_CUDA(cudaMemcpyAsync(a->ckpt[size_t(n / every)], s->q[s->cur], bytes, cudaMemcpyDeviceToDevice, s->stream));
    a->k_step[size_t(n)] = s->steps;
    bbw_status st = bbw_step(s, dt, 1);
    if (st != BBW_OK) return st;
    if (a->nrec > 0)
      sample_kernel<real><<<int((a->nrec + threads - 1) / threads), threads, 0, s->stream>>>(
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
  const size_t nf = size_t(K) * Np, ns = 4 * nf * sizeof(real), bytes = s->nstate_internal() * sizeof(real);
  for (void** b : {&a->qb, &a->rb, &a->y, &a->z, &a->v}) {
    st = dalloc(b, ns);
    if (st != BBW_OK) return st;
  }
  for (void** b : {&a->yi, &a->zi, &a->rs}) {
    st = dalloc(b, bytes);
    if (st != BBW_OK) return st;
  }
  st = dalloc(&a->yt, nf * sizeof(real));
  if (st == BBW_OK) st = dalloc(&a->gc, size_t(K) * Mp * sizeof(real));
  if (st == BBW_OK) st = dalloc(&a->u, size_t(Mp) * nf * sizeof(real));
  if (st != BBW_OK) return st;
  if (!a->blas) {
    BBW_BLAS(cublasCreate(&a->blas));
    BBW_BLAS(cublasSetMathMode(a->blas, CUBLAS_PEDANTIC_MATH));
  }
  BBW_BLAS(cublasSetStream(a->blas, s->stream));
  if (st != BBW_OK) return st;
  {  // the current c^2 of the solver, [K][Mp] in the internal element order
    std::vector<double> c2u(s->c2.size());
    for (int64_t e = 0; e < K; ++e)
      for (int b = 0; b < Mp; ++b) c2u[size_t(e) * Mp + b] = s->c2[size_t(s->user(e)) * Mp + b];
    st = upload_real<real>(c2u, &a->d_c2u);
    if (st != BBW_OK) return st;
  }
  while (a->seg.size() > size_t(a->every) * 5) {  // the five stage inputs of each step of a segment
    if (a->seg.back()) cudaFree(a->seg.back());
    a->seg.pop_back();
  }
  a->seg.resize(size_t(a->every) * 5, nullptr);
  for (auto& b : a->seg) {
    st = dalloc(&b, bytes);
    if (st != BBW_OK) return st;
  }
  if (a->d_g) cudaFree(a->d_g);
  a->d_g = nullptr;
  if (a->nrec > 0 && g) {
    const size_t ng = size_t(a->nsteps) * a->nrec;
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_g), ng * sizeof(double)));
    BBW_CUDA(cudaMemcpy(a->d_g, g, ng * sizeof(double), cudaMemcpyHostToDevice));
  }
  cudaStream_t sm = s->stream;
  BBW_CUDA(cudaMemsetAsync(a->qb, 0, ns, sm));
  BBW_CUDA(cudaMemsetAsync(a->rb, 0, ns, sm));
  BBW_CUDA(cudaMemsetAsync(a->gc, 0, size_t(K) * Mp * sizeof(real), sm));
  const double dt = a->dt;
  const int64_t nseg = int64_t(a->ckpt.size());
  for (int64_t k = nseg - 1; k >= 0; --k) {
    const int64_t n0 = k * a->every, n1 = std::min(a->nsteps, n0 + a->every);
    // the stage inputs of every step of the segment, from its checkpoint
    BBW_CUDA(cudaMemcpyAsync(a->seg[0], a->ckpt[size_t(k)], bytes, cudaMemcpyDeviceToDevice, sm));
    for (int64_t n = n0; n < n1; ++n) {
      const size_t b5 = size_t(n - n0) * 5;
      for (int sg = 0; sg < 5; ++sg) {
        if (sg == 4 && n + 1 == n1) break;  // the segment's final state is not needed
        void* out = sg < 4 ? a->seg[b5 + sg + 1] : a->seg[b5 + 5];
        st = forward_stage<real>(s, a->seg[b5 + sg], out, a->rs, sg, dt, a->k_step[size_t(n)]);
        if (st != BBW_OK) return st;
      }
    }
    for (int64_t n = n1 - 1; n >= n0; --n) {
      // cotangent of the traces after step n
      if (a->d_g) {
        receiver_adjoint_kernel<real><<<1, 256, 0, sm>>>(static_cast<real*>(a->qb), K, a->nrec, a->d_rec_elem,
                                                         static_cast<const real*>(a->d_rec_vec),
                                                         a->d_g + size_t(n) * a->nrec, Np);
        BBW_CUDA(cudaGetLastError());
      }
      const size_t b5 = size_t(n - n0) * 5;
      for (int sg = 4; sg >= 0; --sg) {
        st = adjoint_stage<real>(s, a, a->seg[b5 + sg], sg, dt, a->k_step[size_t(n)]);
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
    std::vector<real> h(4 * nf);
    BBW_CUDA(cudaMemcpy(h.data(), a->qb, h.size() * sizeof(real), cudaMemcpyDeviceToHost));
    for (int f = 0; f < 4; ++f)
      for (int64_t e = 0; e < K; ++e)
        for (int i = 0; i < Np; ++i)
          grad_q0[(size_t(f) * K + size_t(s->user(e))) * Np + i] = double(h[(size_t(f) * K + e) * Np + i]);
  }
  return BBW_OK;
}

}  // namespace

namespace bbw {

void free_adjoint(bbw_solver* s) {
  AdjointData* a = s->adj;
  if (!a) return;
  free_run(a, true);
  for (void* p : {static_cast<void*>(a->d_rec_elem), a->d_rec_vec, a->d_minv, a->d_mass, a->d_tw, a->d_vol, a->d_ivol,
                  a->d_c2u, a->qb, a->rb, a->y, a->z, a->v, a->yt, a->gc, a->yi, a->zi, a->rs, a->qs[0], a->qs[1],
                  a->qs[2], a->qs[3], a->qs[4], static_cast<void*>(a->d_g), a->u})
    if (p) cudaFree(p);
  if (a->blas) cublasDestroy(a->blas);
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
  std::vector<double> vec(static_cast<size_t>(nrec) * s->Np, 0.0);
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
    for (size_t i = 0; i < A.size(); ++i) {
      double b = bbw::factorial(s->N) /
                 (bbw::factorial(A[i][0]) * bbw::factorial(A[i][1]) * bbw::factorial(A[i][2]) * bbw::factorial(A[i][3]));
      for (int m = 0; m < 4; ++m) b *= std::pow(std::max(lam[m], 0.0), A[i][m]);
      vec[size_t(r) * s->Np + i] = b;
    }
  }
  if (a->d_rec_elem) cudaFree(a->d_rec_elem);
  if (a->d_rec_vec) cudaFree(a->d_rec_vec);
  a->d_rec_elem = nullptr;
  a->d_rec_vec = nullptr;
  a->nrec = nrec;
  a->rec_elem = el;
  free_run(a);
  if (nrec > 0) {
    BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->d_rec_elem), size_t(nrec) * sizeof(int64_t)));
    std::vector<int64_t> slots(el.size());
    for (size_t r = 0; r < el.size(); ++r) slots[r] = s->slot(el[r]);  // internal element order
    BBW_CUDA(cudaMemcpy(a->d_rec_elem, slots.data(), size_t(nrec) * sizeof(int64_t), cudaMemcpyHostToDevice));
    bbw_status st = s->prec == 64 ? upload_real<double>(vec, &a->d_rec_vec) : upload_real<float>(vec, &a->d_rec_vec);
    if (st != BBW_OK) return st;
  }
  if (elems) std::copy(el.begin(), el.end(), elems);
  return BBW_OK;
}

bbw_status bbw_record(bbw_solver* s, double dt, int64_t nsteps, int64_t checkpoint_every, double* traces) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (nsteps < 1 || checkpoint_every < 1) return fail(BBW_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
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
