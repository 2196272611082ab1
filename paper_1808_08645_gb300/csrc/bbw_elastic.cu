// bbw_elastic.cu -- host side of the elastic solver (bbw_elastic_* in
// include/bbwadg.h): media and state management and the stage launches of
// bbw_elastic.cuh. The mesh (geometry, connectivity, element renumbering)
// and the operator tables come from an acoustic solver object created with
// the same mesh, whose own state buffers are released.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "bbw_common.h"
#include "bbw_elastic.cuh"
#include "bbw_elastic_ops.h"
#include "bbw_solver.h"
#include "bbwadg.h"

using bbw::fail;

struct bbw_elastic {
  bbw_solver* m = nullptr;  // mesh, renumbering, tables, stream, status word
  const bbw::ElasticOps* ops = nullptr;
  int V = 1;
  int64_t G = 0;
  int grid = 1;
  void* q[2] = {nullptr, nullptr};
  void* res = nullptr;
  void* d_media = nullptr;  // [G][3][Mp][V]
  void* d_geom = nullptr;   // [G][9][V]
  int32_t* d_conn = nullptr;  // [G][4][V]
  void* d_stage = nullptr;  // FP64 user-layout staging of host state transfers
  std::vector<double> media;  // [3][K][Mp], caller's element order
  int cur = 0;
  double t = 0.0;
  int64_t stages = 0;
  double tau_v = 1.0, tau_s = 1.0;
  double rk_a[5] = {}, rk_b[5] = {};
  size_t nuser() const { return size_t(9) * size_t(m->K) * size_t(m->Np); }
  size_t ninternal() const { return size_t(9) * size_t(G) * V * m->Np; }
  size_t rsz() const { return m->prec == 64 ? 8 : 4; }
};

namespace {

// [F][K][Np] FP64 (caller's element order) <-> [G][F][Np][V] of the solver
// precision; internal slot e holds the caller's element perm[e]. Padding
// entries of the internal layout are set to zero.
template <typename From, typename real>
__global__ void elastic_to_internal(const From* __restrict__ src, real* __restrict__ dst, int64_t K, int Np, int V,
                                    int F, const int32_t* __restrict__ perm, size_t n) {
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n; x += size_t(gridDim.x) * blockDim.x) {
    const int v = int(x % V);
    const size_t r = x / V;
    const int i = int(r % Np);
    const size_t r2 = r / Np;
    const int f = int(r2 % F);
    const int64_t e = int64_t(r2 / F) * V + v;
    dst[x] = e < K ? real(src[(size_t(f) * K + (perm ? perm[e] : e)) * Np + i]) : real(0);
  }
}

template <typename real, typename To>
__global__ void elastic_to_user(const real* __restrict__ src, To* __restrict__ dst, int64_t K, int Np, int V,
                                int F, const int32_t* __restrict__ inv) {
  const size_t n = size_t(F) * K * Np;
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n; x += size_t(gridDim.x) * blockDim.x) {
    const int i = int(x % Np);
    const size_t r = x / Np;
    const int64_t eu = int64_t(r % K);
    const int f = int(r / K);
    const int64_t e = inv ? inv[eu] : eu;
    dst[x] = To(src[((size_t(e / V) * F + f) * Np + i) * V + size_t(e % V)]);
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int conv_blocks(size_t n) { return int(std::min<size_t>((n + 255) / 256, size_t(sm_count()) * 16)); }

void free_elastic(bbw_elastic* s) {
  if (!s) return;
  for (void* p : {s->q[0], s->q[1], s->res, s->d_media, s->d_geom, static_cast<void*>(s->d_conn), s->d_stage})
    if (p) cudaFree(p);
  if (s->m) bbw_destroy(s->m);
  delete s;
}

template <typename real>
bbw_status upload_media(bbw_elastic* s) {
  bbw_solver* m = s->m;
  const int Mp = m->Mp, V = s->V;
  std::vector<real> h(size_t(s->G) * 3 * Mp * V);
  for (int64_t e = 0; e < s->G * V; ++e)
    for (int w = 0; w < 3; ++w)
      for (int b = 0; b < Mp; ++b)
        h[((size_t(e / V) * 3 + w) * Mp + b) * V + size_t(e % V)] =
            real(e < m->K ? s->media[(size_t(w) * m->K + size_t(m->user(e))) * Mp + b] : 1.0);
  BBW_CUDA(cudaMemcpyAsync(s->d_media, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice, m->stream));
  BBW_CUDA(cudaStreamSynchronize(m->stream));
  return BBW_OK;
}

template <typename real>
bbw_status upload_mesh(bbw_elastic* s) {
  bbw_solver* m = s->m;
  const int V = s->V;
  // geometry [G][9][V]: d lambda_m / d x for m = 1..3; padding: the unit tetrahedron
  std::vector<double> g9(size_t(m->K) * 9);
  for (int64_t e = 0; e < m->K; ++e)
    for (int c = 0; c < 9; ++c) g9[size_t(e) * 9 + c] = m->grad[size_t(e) * 12 + 3 + c];
  {
    std::vector<real> h(size_t(s->G) * 9 * V);
    for (int64_t e = 0; e < s->G * V; ++e)
      for (int c = 0; c < 9; ++c)
        h[(size_t(e / V) * 9 + c) * V + size_t(e % V)] =
            real(e < m->K ? g9[size_t(m->user(e)) * 9 + c] : (c % 4 == 0 ? 1.0 : 0.0));
    BBW_CUDA(cudaMemcpy(s->d_geom, h.data(), h.size() * sizeof(real), cudaMemcpyHostToDevice));
  }
  // connectivity [G][4][V]: (internal neighbour slot << 5) | (its face << 3) | orientation; -1: wall
  std::vector<int32_t> conn(size_t(s->G) * 4 * V, -1);
  for (int64_t e = 0; e < m->K; ++e)
    for (int f = 0; f < 4; ++f) {
      const size_t i = size_t(m->user(e)) * 4 + f;
      conn[(size_t(e / V) * 4 + f) * V + size_t(e % V)] =
          m->etoe[i] < 0 ? -1
                         : (int32_t(m->slot(m->etoe[i])) << 5) | (int32_t(m->etof[i]) << 3) | int32_t(m->fperm[i]);
    }
  BBW_CUDA(cudaMemcpy(s->d_conn, conn.data(), conn.size() * 4, cudaMemcpyHostToDevice));
  return BBW_OK;
}

template <typename real>
bbw_status launch(bbw_elastic* s, int stage, double dt) {
  bbw_solver* m = s->m;
  bbw::ElasticParams<real> P;
  P.qin = static_cast<const real*>(s->q[s->cur]);
  P.qout = static_cast<real*>(s->q[1 - s->cur]);
  P.res = static_cast<real*>(s->res);
  P.media = static_cast<const real*>(s->d_media);
  P.geom = static_cast<const real*>(s->d_geom);
  P.conn = s->d_conn;
  P.tables = m->op->tables;
  P.G = s->G;
  P.a = real(s->rk_a[stage]);
  P.b = real(s->rk_b[stage]);
  P.dt = real(dt);
  P.tau_v = real(s->tau_v);
  P.tau_s = real(s->tau_s);
  P.status = m->d_status;
  BBW_CUDA(s->ops->launch(m->M, m->prec == 64, &P, s->grid, m->stream));
  s->cur = 1 - s->cur;
  s->stages += 1;
  if (stage == 4) s->t += dt;
  return BBW_OK;
}

// user layout [9][K][Np] of precision src_prec (device) -> internal layout
template <typename From>
void to_internal_t(bbw_elastic* s, const From* src, void* dst) {
  bbw_solver* m = s->m;
  const size_t n = s->ninternal();
  if (m->prec == 64)
    elastic_to_internal<From, double><<<conv_blocks(n), 256, 0, m->stream>>>(src, static_cast<double*>(dst), m->K,
                                                                              m->Np, s->V, 9, m->d_perm, n);
  else
    elastic_to_internal<From, float><<<conv_blocks(n), 256, 0, m->stream>>>(src, static_cast<float*>(dst), m->K,
                                                                             m->Np, s->V, 9, m->d_perm, n);
}

bbw_status to_internal(bbw_elastic* s, const void* src, int src_prec, void* dst) {
  if (src_prec == 64)
    to_internal_t(s, static_cast<const double*>(src), dst);
  else
    to_internal_t(s, static_cast<const float*>(src), dst);
  BBW_CUDA(cudaGetLastError());
  return BBW_OK;
}

// internal layout -> user layout [9][K][Np] of precision dst_prec (device)
template <typename To>
void to_user_t(bbw_elastic* s, const void* src, To* dst) {
  bbw_solver* m = s->m;
  const size_t n = s->nuser();
  if (m->prec == 64)
    elastic_to_user<double, To><<<conv_blocks(n), 256, 0, m->stream>>>(static_cast<const double*>(src), dst, m->K,
                                                                        m->Np, s->V, 9, m->d_inv);
  else
    elastic_to_user<float, To><<<conv_blocks(n), 256, 0, m->stream>>>(static_cast<const float*>(src), dst, m->K,
                                                                       m->Np, s->V, 9, m->d_inv);
}

bbw_status to_user(bbw_elastic* s, const void* src, void* dst, int dst_prec) {
  if (dst_prec == 64)
    to_user_t(s, src, static_cast<double*>(dst));
  else
    to_user_t(s, src, static_cast<float*>(dst));
  BBW_CUDA(cudaGetLastError());
  return BBW_OK;
}

}  // namespace

extern "C" {

bbw_status bbw_elastic_create(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N, int M,
                              int precision, void* cuda_stream, bbw_elastic** out) {
  if (!out) return fail(BBW_ERR_ARG, "out is NULL");
  *out = nullptr;
  auto* s = new bbw_elastic();
  std::vector<std::pair<int64_t, int64_t>> ranges = {{0, K}};
  bbw_status st = bbw::create_solver(nverts, vxyz, K, etov, N, M, precision, cuda_stream, &ranges, &s->m);
  if (st != BBW_OK) {
    delete s;
    return st;
  }
  bbw_solver* m = s->m;
  // the acoustic state, c^2 and layout buffers are not used
  for (void** p : {&m->q[0], &m->q[1], &m->res, &m->d_c2, &m->d_geom, reinterpret_cast<void**>(&m->d_conn)}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  s->ops = bbw::elastic_ops_for(N);
  int team = 0, gpc = 1, per_sm = 0;
  s->ops->shape(M, precision == 64, &team, &s->V, &gpc);
  cudaError_t err = s->ops->prepare(M, precision == 64, &per_sm);
  if (err != cudaSuccess) {
    free_elastic(s);
    return fail(BBW_ERR_CUDA, std::string("elastic kernel set-up: ") + cudaGetErrorString(err));
  }
  s->G = (K + s->V - 1) / s->V;
  const int64_t tiles = (s->G + gpc - 1) / gpc;
  s->grid = int(std::min<int64_t>(tiles, int64_t(std::max(1, per_sm)) * sm_count()));
  double c[5];
  bbw_lsrk_coeffs(s->rk_a, s->rk_b, c);
  const size_t rs = s->rsz();
  const size_t ng = size_t(s->G) * s->V;
  auto alloc = [&](void** p, size_t bytes) {
    return cudaMalloc(p, bytes) == cudaSuccess && cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  const bool ok = alloc(&s->q[0], s->ninternal() * rs) && alloc(&s->q[1], s->ninternal() * rs) &&
                  alloc(&s->res, s->ninternal() * rs) && alloc(&s->d_media, ng * 3 * m->Mp * rs) &&
                  alloc(&s->d_geom, ng * 9 * rs) && alloc(reinterpret_cast<void**>(&s->d_conn), ng * 16) &&
                  alloc(&s->d_stage, s->nuser() * 8);
  if (!ok) {
    std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(cudaGetLastError());
    free_elastic(s);
    return fail(BBW_ERR_CUDA, msg);
  }
  st = precision == 64 ? upload_mesh<double>(s) : upload_mesh<float>(s);
  if (st == BBW_OK) {
    s->media.assign(size_t(3) * K * m->Mp, 1.0);
    st = precision == 64 ? upload_media<double>(s) : upload_media<float>(s);
  }
  if (st != BBW_OK) {
    free_elastic(s);
    return st;
  }
  *out = s;
  return BBW_OK;
}

void bbw_elastic_destroy(bbw_elastic* s) {
  if (s && s->m && s->m->stream)
    cudaStreamSynchronize(s->m->stream);
  else if (s)
    cudaDeviceSynchronize();
  free_elastic(s);
}

bbw_status bbw_elastic_info(const bbw_elastic* s, int64_t* K, int* N, int* M, int* Np, int* Mp, int* precision) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return bbw_info(s->m, K, N, M, Np, Mp, precision);
}

bbw_status bbw_elastic_set_media(bbw_elastic* s, const double* rho_inv, const double* lam, const double* mu) {
  if (!s || !rho_inv || !lam || !mu) return fail(BBW_ERR_ARG, "NULL argument");
  bbw_solver* m = s->m;
  const size_t n = size_t(m->K) * m->Mp;
  for (size_t i = 0; i < n; ++i) {
    if (!(rho_inv[i] > 0.0) || !std::isfinite(rho_inv[i]))
      return fail(BBW_ERR_NONPOS_C2, "a rho^{-1} coefficient is <= 0 or not finite");
    if (!(lam[i] >= 0.0) || !std::isfinite(lam[i]) || !(mu[i] >= 0.0) || !std::isfinite(mu[i]))
      return fail(BBW_ERR_NONPOS_C2, "a lambda or mu coefficient is < 0 or not finite");
  }
  std::memcpy(s->media.data(), rho_inv, n * 8);
  std::memcpy(s->media.data() + n, lam, n * 8);
  std::memcpy(s->media.data() + 2 * n, mu, n * 8);
  return m->prec == 64 ? upload_media<double>(s) : upload_media<float>(s);
}

bbw_status bbw_elastic_set_params(bbw_elastic* s, double tau_v, double tau_s) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (!std::isfinite(tau_v) || !std::isfinite(tau_s) || tau_v < 0.0 || tau_s < 0.0)
    return fail(BBW_ERR_ARG, "penalty parameters must be finite and >= 0");
  s->tau_v = tau_v;
  s->tau_s = tau_s;
  return BBW_OK;
}

bbw_status bbw_elastic_set_state(bbw_elastic* s, const double* q, const double* res, double t) {
  if (!s || !q) return fail(BBW_ERR_ARG, "NULL argument");
  if (!std::isfinite(t)) return fail(BBW_ERR_ARG, "t is not finite");
  bbw_solver* m = s->m;
  const size_t bytes = s->nuser() * 8;
  double* d = static_cast<double*>(s->d_stage);
  BBW_CUDA(cudaMemcpyAsync(d, q, bytes, cudaMemcpyHostToDevice, m->stream));
  bbw_status st = to_internal(s, d, 64, s->q[s->cur]);
  if (st != BBW_OK) return st;
  if (res) {
    BBW_CUDA(cudaMemcpyAsync(d, res, bytes, cudaMemcpyHostToDevice, m->stream));
    st = to_internal(s, d, 64, s->res);
    if (st != BBW_OK) return st;
  } else {
    BBW_CUDA(cudaMemsetAsync(s->res, 0, s->ninternal() * s->rsz(), m->stream));
  }
  BBW_CUDA(cudaStreamSynchronize(m->stream));
  s->t = t;
  s->stages = 0;
  return BBW_OK;
}

bbw_status bbw_elastic_get_state(bbw_elastic* s, double* q, double* res, double* t) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  bbw_status st = bbw::check_status(s->m);
  if (st != BBW_OK) return st;
  bbw_solver* m = s->m;
  const size_t bytes = s->nuser() * 8;
  double* d = static_cast<double*>(s->d_stage);
  if (q) {
    st = to_user(s, s->q[s->cur], d, 64);
    if (st != BBW_OK) return st;
    BBW_CUDA(cudaMemcpyAsync(q, d, bytes, cudaMemcpyDeviceToHost, m->stream));
    BBW_CUDA(cudaStreamSynchronize(m->stream));
  }
  if (res) {
    st = to_user(s, s->res, d, 64);
    if (st != BBW_OK) return st;
    BBW_CUDA(cudaMemcpyAsync(res, d, bytes, cudaMemcpyDeviceToHost, m->stream));
    BBW_CUDA(cudaStreamSynchronize(m->stream));
  }
  if (t) *t = s->t;
  return BBW_OK;
}

bbw_status bbw_elastic_set_state_device(bbw_elastic* s, const void* q, const void* res, int dtype, double t) {
  if (!s || !q) return fail(BBW_ERR_ARG, "NULL argument");
  if (dtype != 32 && dtype != 64) return fail(BBW_ERR_ARG, "dtype must be 32 or 64");
  if (!std::isfinite(t)) return fail(BBW_ERR_ARG, "t is not finite");
  bbw_status st = to_internal(s, q, dtype, s->q[s->cur]);
  if (st != BBW_OK) return st;
  if (res) {
    st = to_internal(s, res, dtype, s->res);
    if (st != BBW_OK) return st;
  } else {
    BBW_CUDA(cudaMemsetAsync(s->res, 0, s->ninternal() * s->rsz(), s->m->stream));
  }
  s->t = t;
  s->stages = 0;
  return BBW_OK;
}

bbw_status bbw_elastic_get_state_device(bbw_elastic* s, void* q, void* res, int dtype) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (dtype != 32 && dtype != 64) return fail(BBW_ERR_ARG, "dtype must be 32 or 64");
  if (q) {
    bbw_status st = to_user(s, s->q[s->cur], q, dtype);
    if (st != BBW_OK) return st;
  }
  if (res) {
    bbw_status st = to_user(s, s->res, res, dtype);
    if (st != BBW_OK) return st;
  }
  return BBW_OK;
}

bbw_status bbw_elastic_stage(bbw_elastic* s, int stage, double dt) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (stage < 0 || stage > 4) return fail(BBW_ERR_ARG, "stage must be in 0..4");
  if (!std::isfinite(dt)) return fail(BBW_ERR_ARG, "dt is not finite");
  return s->m->prec == 64 ? launch<double>(s, stage, dt) : launch<float>(s, stage, dt);
}

bbw_status bbw_elastic_step(bbw_elastic* s, double dt, int64_t nsteps) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (nsteps < 0) return fail(BBW_ERR_ARG, "nsteps < 0");
  for (int64_t i = 0; i < nsteps; ++i)
    for (int st = 0; st < 5; ++st) {
      bbw_status r = bbw_elastic_stage(s, st, dt);
      if (r != BBW_OK) return r;
    }
  return BBW_OK;
}

bbw_status bbw_elastic_cfl_dt(const bbw_elastic* s, double cfl, double* dt) {
  if (!s || !dt) return fail(BBW_ERR_ARG, "NULL argument");
  if (!(cfl > 0.0)) return fail(BBW_ERR_ARG, "cfl must be > 0");
  const bbw_solver* m = s->m;
  const size_t n = size_t(m->K) * m->Mp;
  // P-wave speed^2 = (lambda + 2 mu) / rho <= max(lambda + 2 mu) max(rho^{-1})
  // on each element (Bernstein coefficients bound the polynomial)
  double cp2 = 0.0, ratio = 0.0;
  for (int64_t e = 0; e < m->K; ++e) {
    double a = 0.0, r = 0.0;
    for (int b = 0; b < m->Mp; ++b) {
      const size_t i = size_t(e) * m->Mp + b;
      a = std::max(a, s->media[n + i] + 2.0 * s->media[2 * n + i]);
      r = std::max(r, s->media[i]);
    }
    cp2 = std::max(cp2, a * r);
    for (int f = 0; f < 4; ++f) {
      const double* g = &m->grad[size_t(e) * 12 + 3 * f];
      ratio = std::max(ratio, 3.0 * std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
    }
  }
  const double cn = (m->N + 1) * (m->N + 3) / 3.0;
  *dt = cfl / (std::sqrt(cp2) * cn * ratio);
  return BBW_OK;
}

bbw_status bbw_elastic_advance(bbw_elastic* s, double T, double cfl, double* dt_used, int64_t* nsteps) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (!(T >= 0.0) || !std::isfinite(T)) return fail(BBW_ERR_ARG, "T must be finite and >= 0");
  double dt = 0.0;
  bbw_status st = bbw_elastic_cfl_dt(s, cfl, &dt);
  if (st != BBW_OK) return st;
  const int64_t n = int64_t(std::ceil(T / dt));
  const double h = n > 0 ? T / double(n) : 0.0;
  if (dt_used) *dt_used = h;
  if (nsteps) *nsteps = n;
  return bbw_elastic_step(s, h, n);
}

bbw_status bbw_elastic_sync(bbw_elastic* s) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return bbw::check_status(s->m);
}

bbw_status bbw_elastic_get_time(const bbw_elastic* s, double* t, int64_t* stages) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (t) *t = s->t;
  if (stages) *stages = s->stages;
  return BBW_OK;
}

}  // extern "C"
