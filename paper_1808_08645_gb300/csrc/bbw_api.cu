// bbw_api.cu -- host side of libbbwadg: mesh setup, constants, state
// management and the C ABI declared in include/bbwadg.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "bbw_common.h"
#include "bbw_ops.h"
#include "bbw_stage.cuh"
#include "bbwadg.h"
#include "bbw_solver.h"

using bbw::fail;
using bbw::OpCache;
using bbw::check_status;
using bbw::ensure_pinned;

namespace {

thread_local std::string g_err;


// ---------------------------------------------------------------------------
// constants

// Eigenvalue of the normalised degree-n Bernstein mass matrix on the
// tetrahedron for modal degree k <= n: (n!)^2 3! / ((n+k+3)! (n-k)!).
// (Lemma 5.2 states M_N is diagonal in a modal basis with one eigenvalue per
// modal degree; this is the closed form of those eigenvalues.)
long double mass_eig(int n, int k) {
  return expl(2.0L * lgammal(n + 1.0L) + logl(6.0L) - lgammal(n + k + 4.0L) - lgammal(n - k + 1.0L));
}

// c_j of Theorem 5.3: in the modal basis the decomposition reads, for each
// modal degree k = 0..N, sum_{j=0}^{N-k} c_j lam^{N-j}_k = lam^{N+M}_k
// (Corollary 1 and Lemma 5.2 with the proof of Theorem 5.3); solved
// top-down from k = N.
void projection_coeffs(int N, int M, double* c) {
  long double cc[bbw::kMaxN + 1] = {};
  for (int k = N; k >= 0; --k) {
    long double s = mass_eig(N + M, k);
    for (int j = 0; j < N - k; ++j) s -= cc[j] * mass_eig(N - j, k);
    cc[N - k] = s / mass_eig(k, k);
  }
  for (int j = 0; j <= N; ++j) c[j] = double(cc[j]);
}

// Carpenter-Kennedy five-stage fourth-order 2N-storage RK coefficients.
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

// Stage times from the equivalent Butcher rows: stage s sees
// q_0 + h sum_{m<s} A[s][m] F_m, A[s][m] = sum_{i=m}^{s-1} b_i prod_{r=m+1}^{i} a_r.
std::array<double, 5> rk_stage_times() {
  std::array<double, 5> c{};
  for (int s = 1; s < 5; ++s) {
    double acc = 0.0;
    for (int m = 0; m < s; ++m)
      for (int i = m; i < s; ++i) {
        double p = kRkB[i];
        for (int r = m + 1; r <= i; ++r) p *= kRkA[r];
        acc += p;
      }
    c[s] = acc;
  }
  return c;
}

double factd(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// multi-indices of degree n in the library order
std::vector<std::array<int, 4>> multi_indices(int n) {
  std::vector<std::array<int, 4>> out;
  for (int l = 0; l <= n; ++l)
    for (int k = 0; k <= n - l; ++k)
      for (int j = 0; j <= n - l - k; ++j) out.push_back({n - j - k - l, j, k, l});
  return out;
}

// Solve (normalised Bernstein mass matrix) x = b by Cholesky, in place.
bool mass_solve(int n, std::vector<double>& b) {
  const auto A = multi_indices(n);
  const int P = int(A.size());
  std::vector<double> L(size_t(P) * P);
  auto coef = [&](const std::array<int, 4>& a) {
    return factd(n) / (factd(a[0]) * factd(a[1]) * factd(a[2]) * factd(a[3]));
  };
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double m = 6.0 / factd(2 * n + 3);
      for (int x = 0; x < 4; ++x) m *= factd(A[i][x] + A[j][x]);
      L[size_t(i) * P + j] = coef(A[i]) * coef(A[j]) * m;
    }
  for (int j = 0; j < P; ++j) {
    double d = L[size_t(j) * P + j];
    for (int k = 0; k < j; ++k) d -= L[size_t(j) * P + k] * L[size_t(j) * P + k];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    L[size_t(j) * P + j] = d;
    for (int i = j + 1; i < P; ++i) {
      double s = L[size_t(i) * P + j];
      for (int k = 0; k < j; ++k) s -= L[size_t(i) * P + k] * L[size_t(j) * P + k];
      L[size_t(i) * P + j] = s / d;
    }
  }
  for (int i = 0; i < P; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[size_t(i) * P + k] * b[k];
    b[i] = s / L[size_t(i) * P + i];
  }
  for (int i = P - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < P; ++k) s -= L[size_t(k) * P + i] * b[k];
    b[i] = s / L[size_t(i) * P + i];
  }
  return true;
}

// ---------------------------------------------------------------------------
// small device helpers

// State layouts: the ABI's [4][K][Np] ("user") and the kernels' grouped
// [G][4][Np][V] ("internal", V elements per group, G = ceil(K / V); entries of
// the padding elements of the last group are zero).
__host__ __device__ inline size_t internal_index(int64_t e, int i, int f, int Np, int V) {
  return ((size_t(e / V) * 4 + f) * Np + i) * V + size_t(e % V);
}

// Internal element slot e holds the caller's element perm[e] (perm NULL:
// the identity); inv is the inverse permutation.
template <typename From, typename To>
__global__ void to_internal_kernel(const From* __restrict__ src, To* __restrict__ dst, int64_t K, int Np, int V,
                                   const int32_t* __restrict__ perm, size_t n_internal) {
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n_internal; x += size_t(gridDim.x) * blockDim.x) {
    // x enumerates the internal layout: decode (g, f, i, v)
    const int v = int(x % V);
    const size_t r = x / V;
    const int i = int(r % Np);
    const size_t r2 = r / Np;
    const int f = int(r2 % 4);
    const int64_t e = int64_t(r2 / 4) * V + v;
    dst[x] = e < K ? To(src[(size_t(f) * K + (perm ? perm[e] : e)) * Np + i]) : To(0);
  }
}

template <typename From, typename To>
__global__ void to_user_kernel(const From* __restrict__ src, To* __restrict__ dst, int64_t K, int Np, int V,
                               const int32_t* __restrict__ inv) {
  const size_t n = size_t(4) * K * Np;
  for (size_t x = blockIdx.x * size_t(blockDim.x) + threadIdx.x; x < n; x += size_t(gridDim.x) * blockDim.x) {
    const int i = int(x % Np);
    const size_t r = x / Np;
    const int64_t e = int64_t(r % K);
    const int f = int(r / K);
    dst[x] = To(src[internal_index(inv ? inv[e] : e, i, f, Np, V)]);
  }
}

template <typename From, typename To>
cudaError_t state_to_internal(const void* src, void* dst, int64_t K, int Np, int V, const int32_t* perm,
                              cudaStream_t s) {
  const size_t n = size_t((K + V - 1) / V) * V * Np * 4;
  const int blocks = int(std::min<size_t>((n + 255) / 256, 152 * 16));
  to_internal_kernel<From, To><<<blocks, 256, 0, s>>>(static_cast<const From*>(src), static_cast<To*>(dst), K, Np, V,
                                                      perm, n);
  return cudaGetLastError();
}

template <typename From, typename To>
cudaError_t state_to_user(const void* src, void* dst, int64_t K, int Np, int V, const int32_t* inv, cudaStream_t s) {
  const size_t n = size_t(4) * K * Np;
  const int blocks = int(std::min<size_t>((n + 255) / 256, 152 * 16));
  to_user_kernel<From, To><<<blocks, 256, 0, s>>>(static_cast<const From*>(src), static_cast<To*>(dst), K, Np, V,
                                                  inv);
  return cudaGetLastError();
}

cudaError_t copy_to_internal_impl(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np,
                                  int V, const int32_t* perm, cudaStream_t s) {
  if (src_prec == 64)
    return dst_prec == 64 ? state_to_internal<double, double>(src, dst, K, Np, V, perm, s)
                          : state_to_internal<double, float>(src, dst, K, Np, V, perm, s);
  return dst_prec == 64 ? state_to_internal<float, double>(src, dst, K, Np, V, perm, s)
                        : state_to_internal<float, float>(src, dst, K, Np, V, perm, s);
}

cudaError_t copy_to_user_impl(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np, int V,
                              const int32_t* inv, cudaStream_t s) {
  if (src_prec == 64)
    return dst_prec == 64 ? state_to_user<double, double>(src, dst, K, Np, V, inv, s)
                          : state_to_user<double, float>(src, dst, K, Np, V, inv, s);
  return dst_prec == 64 ? state_to_user<float, double>(src, dst, K, Np, V, inv, s)
                        : state_to_user<float, float>(src, dst, K, Np, V, inv, s);
}

std::mutex g_cache_mu;
std::map<std::tuple<int, int, int, int>, OpCache> g_cache;

bbw_status get_tables(int N, int M, int prec, OpCache** out) {
  int dev = 0;
  BBW_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_cache_mu);
  auto key = std::make_tuple(dev, N, M, prec);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = &it->second;
    return BBW_OK;
  }
  const bbw::KernelOps* ops = bbw::ops_for(N);
  const bool dbl = prec == 64;
  double cj[bbw::kMaxN + 1];
  projection_coeffs(N, M, cj);
  const size_t bytes = ops->table_bytes(M, dbl);
  std::vector<unsigned char> host(bytes, 0);
  ops->build_tables(M, dbl, cj, host.data());
  OpCache c;
  BBW_CUDA(ops->prepare(M, dbl, &c.per_sm_stage, &c.per_sm_wadg));
  BBW_CUDA(cudaMalloc(&c.tables, bytes));
  BBW_CUDA(cudaMemcpy(c.tables, host.data(), bytes, cudaMemcpyHostToDevice));
  auto res = g_cache.emplace(key, c);
  *out = &res.first->second;
  return BBW_OK;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

namespace bbw {
void set_last_error(const char* msg) { g_err = msg; }
cudaError_t copy_to_internal(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np, int V,
                             const int32_t* perm, cudaStream_t s) {
  return copy_to_internal_impl(src, src_prec, dst, dst_prec, K, Np, V, perm, s);
}
double factorial(int n) { return factd(n); }
std::vector<std::array<int, 4>> lattice(int n) { return multi_indices(n); }
bool solve_mass(int n, std::vector<double>& b) { return mass_solve(n, b); }
cudaError_t copy_to_user(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np, int V,
                         const int32_t* inv, cudaStream_t s) {
  return copy_to_user_impl(src, src_prec, dst, dst_prec, K, Np, V, inv, s);
}
}  // namespace bbw

// ---------------------------------------------------------------------------
// solver object


namespace {

void free_solver(bbw_solver* s) {
  if (!s) return;
  bbw::free_adjoint(s);
  for (void* p : {s->q[0], s->q[1], s->res, s->d_c2, s->d_geom, static_cast<void*>(s->d_conn), s->d_src,
                  static_cast<void*>(s->d_src_groups), static_cast<void*>(s->d_src_slots),
                  static_cast<void*>(s->d_src_ser), static_cast<void*>(s->d_src_amp), s->d_stage,
                  static_cast<void*>(s->d_perm),
                  static_cast<void*>(s->d_inv),
                  static_cast<void*>(s->d_status)})
    if (p) cudaFree(p);
  if (s->pinned) cudaFreeHost(s->pinned);
  delete s;
}


// host doubles -> device buffer of the solver precision, through pinned memory
bbw_status upload(bbw_solver* s, const double* src, void* dst, size_t n) {
  bbw_status st = ensure_pinned(s, n * 8);
  if (st != BBW_OK) return st;
  if (s->prec == 64) {
    std::memcpy(s->pinned, src, n * 8);
  } else {
    float* p = static_cast<float*>(s->pinned);
    for (size_t i = 0; i < n; ++i) p[i] = float(src[i]);
  }
  BBW_CUDA(cudaMemcpyAsync(dst, s->pinned, n * s->rsz(), cudaMemcpyHostToDevice, s->stream));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  return BBW_OK;
}

bbw_status ensure_stage(bbw_solver* s) {
  const size_t bytes = s->nstate() * sizeof(double);
  if (s->d_stage_bytes >= bytes) return BBW_OK;
  if (s->d_stage) cudaFree(s->d_stage);
  s->d_stage = nullptr;
  s->d_stage_bytes = 0;
  BBW_CUDA(cudaMalloc(&s->d_stage, bytes));
  s->d_stage_bytes = bytes;
  return BBW_OK;
}

// host [4][K][Np] doubles -> device grouped state of the solver precision:
// the array is copied as it is and regrouped (and rounded) on the device
bbw_status upload_state(bbw_solver* s, const double* src, void* dst) {
  bbw_status st = ensure_stage(s);
  if (st != BBW_OK) return st;
  BBW_CUDA(cudaMemcpyAsync(s->d_stage, src, s->nstate() * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  BBW_CUDA(bbw::copy_to_internal(s->d_stage, 64, dst, s->prec, s->K, s->Np, s->V, s->d_perm, s->stream));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  return BBW_OK;
}

bbw_status download_state(bbw_solver* s, const void* src, double* dst) {
  bbw_status st = ensure_stage(s);
  if (st != BBW_OK) return st;
  BBW_CUDA(bbw::copy_to_user(src, s->prec, s->d_stage, 64, s->K, s->Np, s->V, s->d_inv, s->stream));
  BBW_CUDA(cudaMemcpyAsync(dst, s->d_stage, s->nstate() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  return BBW_OK;
}

// host [K][W] doubles -> device [G][W][V] (padding elements get pad)
bbw_status upload_grouped(bbw_solver* s, const double* src, int W, double pad, void* dst) {
  const size_t n = size_t(s->G) * W * s->V;
  bbw_status st = ensure_pinned(s, n * 8);
  if (st != BBW_OK) return st;
  const int V = s->V;
  auto fill = [&](auto* p) {
    using T = std::remove_pointer_t<decltype(p)>;
    for (int64_t e = 0; e < s->G * V; ++e)
      for (int w = 0; w < W; ++w)
        p[(size_t(e / V) * W + w) * V + size_t(e % V)] = T(e < s->K ? src[size_t(s->user(e)) * W + w] : pad);
  };
  if (s->prec == 64)
    fill(static_cast<double*>(s->pinned));
  else
    fill(static_cast<float*>(s->pinned));
  BBW_CUDA(cudaMemcpyAsync(dst, s->pinned, n * s->rsz(), cudaMemcpyHostToDevice, s->stream));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  return BBW_OK;
}


// connectivity by sorting face keys (sorted global vertex triples)
bbw_status build_connectivity(bbw_solver* s) {
  const int64_t K = s->K;
  struct FaceRec {
    int64_t a, b, c;
    int64_t e;
    int f;
  };
  std::vector<FaceRec> faces;
  faces.reserve(size_t(K) * 4);
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      int64_t v[3];
      for (int x = 0; x < 3; ++x) v[x] = s->etov[size_t(e) * 4 + bbw::kFaceVerts[f][x]];
      std::sort(v, v + 3);
      faces.push_back({v[0], v[1], v[2], e, f});
    }
  std::sort(faces.begin(), faces.end(), [](const FaceRec& x, const FaceRec& y) {
    return std::tie(x.a, x.b, x.c, x.e, x.f) < std::tie(y.a, y.b, y.c, y.e, y.f);
  });
  s->etoe.assign(size_t(K) * 4, -1);
  s->etof.assign(size_t(K) * 4, -1);
  s->fperm.assign(size_t(K) * 4, -1);
  auto same = [](const FaceRec& x, const FaceRec& y) { return x.a == y.a && x.b == y.b && x.c == y.c; };
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && same(faces[i], faces[j])) ++j;
    if (j - i > 2) return fail(BBW_ERR_MESH, "a face is shared by more than two elements");
    if (j - i == 2) {
      const FaceRec& x = faces[i];
      const FaceRec& y = faces[i + 1];
      if (x.e == y.e) return fail(BBW_ERR_MESH, "an element repeats a face");
      for (int side = 0; side < 2; ++side) {
        const FaceRec& me = side ? y : x;
        const FaceRec& nb = side ? x : y;
        int64_t G[3], H[3];
        for (int q = 0; q < 3; ++q) {
          G[q] = s->etov[size_t(me.e) * 4 + bbw::kFaceVerts[me.f][q]];
          H[q] = s->etov[size_t(nb.e) * 4 + bbw::kFaceVerts[nb.f][q]];
        }
        int code = -1;
        for (int c = 0; c < 6 && code < 0; ++c)
          if (G[0] == H[bbw::kPerm[c][0]] && G[1] == H[bbw::kPerm[c][1]] && G[2] == H[bbw::kPerm[c][2]]) code = c;
        if (code < 0) return fail(BBW_ERR_MESH, "face vertex mismatch");
        const size_t slot = size_t(me.e) * 4 + me.f;
        s->etoe[slot] = int32_t(nb.e);
        s->etof[slot] = int8_t(nb.f);
        s->fperm[slot] = int8_t(code);
      }
    }
    i = j;
  }
  return BBW_OK;
}

bbw_status build_geometry(bbw_solver* s) {
  const int64_t K = s->K;
  s->grad.assign(size_t(K) * 12, 0.0);
  s->vol.assign(size_t(K), 0.0);
  for (int64_t e = 0; e < K; ++e) {
    double X[4][3];
    for (int v = 0; v < 4; ++v)
      for (int d = 0; d < 3; ++d) X[v][d] = s->vxyz[size_t(s->etov[size_t(e) * 4 + v]) * 3 + d];
    // J columns: v1-v0, v2-v0, v3-v0; lambda_{1..3} = J^{-1}(x - v0)
    double J[3][3];
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) J[d][c] = X[c + 1][d] - X[0][d];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double scale = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) scale = std::max(scale, std::fabs(J[d][c]));
    if (!(det > 1e-14 * scale * scale * scale) || !std::isfinite(det))
      return fail(BBW_ERR_MESH, "element " + std::to_string(e) + " is inverted or degenerate");
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double* g = &s->grad[size_t(e) * 12];
    for (int m = 1; m <= 3; ++m)
      for (int d = 0; d < 3; ++d) g[3 * m + d] = inv[m - 1][d];
    for (int d = 0; d < 3; ++d) g[d] = -(g[3 + d] + g[6 + d] + g[9 + d]);
    s->vol[size_t(e)] = det / 6.0;
  }
  return BBW_OK;
}

// validate the mesh, then geometry and connectivity (host only)
bbw_status setup_mesh(bbw_solver* s, int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N) {
  for (int64_t i = 0; i < K * 4; ++i)
    if (etov[i] < 0 || etov[i] >= nverts) return fail(BBW_ERR_MESH, "vertex id out of range");
  for (int64_t i = 0; i < nverts * 3; ++i)
    if (!std::isfinite(vxyz[i])) return fail(BBW_ERR_MESH, "non-finite vertex coordinate");
  s->N = N;
  s->K = K;
  s->Np = bbw::np3(N);
  s->Nfp = bbw::np2(N);
  s->ops = bbw::ops_for(N);
  s->vxyz.assign(vxyz, vxyz + nverts * 3);
  s->etov.assign(etov, etov + K * 4);
  for (int64_t e = 0; e < K; ++e) {
    const int64_t* v = etov + e * 4;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (v[a] == v[b]) return fail(BBW_ERR_MESH, "element " + std::to_string(e) + " repeats a vertex");
  }
  bbw_status st = build_geometry(s);
  if (st == BBW_OK) st = build_connectivity(s);
  return st;
}

template <typename real>
bbw_status upload_geometry(bbw_solver* s) {
  // [G][9][V]; padding elements of the last group get the unit tetrahedron
  // (grad lambda_m = e_m), whose results are never read back
  const int V = s->V;
  std::vector<real> geom(size_t(s->G) * 9 * V);
  for (int64_t e = 0; e < s->G * V; ++e)
    for (int c = 0; c < 9; ++c)
      geom[(size_t(e / V) * 9 + c) * V + size_t(e % V)] =
          real(e < s->K ? s->grad[size_t(s->user(e)) * 12 + 3 + c] : (c % 4 == 0 ? 1.0 : 0.0));
  BBW_CUDA(cudaMemcpy(s->d_geom, geom.data(), geom.size() * sizeof(real), cudaMemcpyHostToDevice));
  return BBW_OK;
}

template <typename real>
bbw_status launch_stage(bbw_solver* s, int stage, double dt) {
  bbw::StageParams<real> P;
  P.qin = static_cast<const real*>(s->q[s->cur]);
  P.qout = static_cast<real*>(s->q[1 - s->cur]);
  P.res = static_cast<real*>(s->res);
  P.c2 = static_cast<const real*>(s->d_c2);
  P.geom = static_cast<const real*>(s->d_geom);
  P.conn = s->d_conn;
  P.tables = s->op->tables;
  P.G = s->G;
  P.a = real(kRkA[stage]);
  P.b = real(kRkB[stage]);
  P.dt = real(dt);
  P.tau_p = real(s->tau_p);
  P.tau_u = real(s->tau_u);
  bbw::set_stage_sources<bbw::StageParams<real>, real>(s, P, s->steps, stage, true);
  P.status = s->d_status;
  P.vout = static_cast<real*>(s->vout);
  BBW_CUDA(s->ops->launch_stage(s->M, s->prec == 64, &P, s->grid_stage, s->stream));
  s->cur = 1 - s->cur;
  s->stages += 1;
  if (stage == 4) {
    s->t += dt;
    s->steps += 1;
  }
  return BBW_OK;
}

}  // namespace

namespace {

// Internal element order for locality: elements sorted by the Morton key of
// their centroids (10 bits per axis over the mesh's bounding box; ties keep
// the caller's order), so that face neighbours are close in memory and their
// traces are more often still in L2 when gathered.
// With ranges, elements are reordered only within each [lo, hi) range (each
// with its own bounding box) and elements outside every range keep their
// place.
bbw_status renumber_elements(bbw_solver* s, const std::vector<std::pair<int64_t, int64_t>>& ranges) {
  const int64_t K = s->K;
  std::vector<double> cen(size_t(K) * 3, 0.0);
  for (int64_t e = 0; e < K; ++e)
    for (int v = 0; v < 4; ++v)
      for (int d = 0; d < 3; ++d) cen[size_t(e) * 3 + d] += 0.25 * s->vxyz[size_t(s->etov[size_t(e) * 4 + v]) * 3 + d];
  auto spread = [](uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
  };
  s->perm.resize(size_t(K));
  for (int64_t e = 0; e < K; ++e) s->perm[size_t(e)] = int32_t(e);
  std::vector<uint64_t> key(static_cast<size_t>(K), 0);
  for (const auto& [r0, r1] : ranges) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t e = r0; e < r1; ++e)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], cen[size_t(e) * 3 + d]);
        hi[d] = std::max(hi[d], cen[size_t(e) * 3 + d]);
      }
    for (int64_t e = r0; e < r1; ++e) {
      uint64_t k = 0;
      for (int d = 0; d < 3; ++d) {
        const double w = hi[d] > lo[d] ? (cen[size_t(e) * 3 + d] - lo[d]) / (hi[d] - lo[d]) : 0.0;
        const uint64_t q = uint64_t(std::min(1023.0, std::max(0.0, std::floor(w * 1024.0))));
        k |= spread(q) << d;
      }
      key[size_t(e)] = k;
    }
    std::stable_sort(s->perm.begin() + r0, s->perm.begin() + r1,
                     [&](int32_t a, int32_t b) { return key[size_t(a)] < key[size_t(b)]; });
  }
  s->inv.resize(size_t(K));
  for (int64_t e = 0; e < K; ++e) s->inv[size_t(s->perm[size_t(e)])] = int32_t(e);
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_perm), size_t(K) * sizeof(int32_t)));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_inv), size_t(K) * sizeof(int32_t)));
  BBW_CUDA(cudaMemcpy(s->d_perm, s->perm.data(), size_t(K) * sizeof(int32_t), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaMemcpy(s->d_inv, s->inv.data(), size_t(K) * sizeof(int32_t), cudaMemcpyHostToDevice));
  return BBW_OK;
}

}  // namespace

namespace bbw {

bbw_status ensure_pinned(bbw_solver* s, size_t bytes) {
  if (s->pinned_bytes >= bytes) return BBW_OK;
  if (s->pinned) cudaFreeHost(s->pinned);
  s->pinned = nullptr;
  s->pinned_bytes = 0;
  BBW_CUDA(cudaMallocHost(&s->pinned, bytes));
  s->pinned_bytes = bytes;
  return BBW_OK;
}

}  // namespace bbw

namespace bbw {

bbw_status check_status(bbw_solver* s) {
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  BBW_CUDA(cudaGetLastError());
  unsigned int st = 0;
  BBW_CUDA(cudaMemcpy(&st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st) {
    BBW_CUDA(cudaMemset(s->d_status, 0, sizeof(unsigned int)));
    if (st & 2u) return fail(BBW_ERR_MESH, "the checked stage kernel met a neighbour or table index out of range");
    return fail(BBW_ERR_NONFINITE, "the stage kernel produced a non-finite value");
  }
  return BBW_OK;
}

}  // namespace bbw

bbw_status bbw::point_source_vector(const bbw_solver* s, const double* xs, int64_t e_begin, int64_t e_end,
                                    int64_t* elem, std::vector<double>* vec) {
  int64_t found = -1;
  double lam[4] = {0, 0, 0, 0};
  for (int64_t e = e_begin; e < e_end && found < 0; ++e) {
    const double* g = &s->grad[size_t(e) * 12];
    const double* v0 = &s->vxyz[size_t(s->etov[size_t(e) * 4]) * 3];
    double l[4];
    bool inside = true;
    for (int m = 0; m < 4; ++m) {
      l[m] = (m == 0 ? 1.0 : 0.0);
      for (int d = 0; d < 3; ++d) l[m] += g[3 * m + d] * (xs[d] - v0[d]);
      inside = inside && l[m] >= -1e-12;
    }
    if (inside) {
      found = e;
      std::memcpy(lam, l, sizeof(lam));
    }
  }
  if (found < 0) return fail(BBW_ERR_ARG, "source point lies outside the mesh");
  const auto A = multi_indices(s->N);
  std::vector<double>& b = *vec;
  b.assign(A.size(), 0.0);
  for (size_t i = 0; i < A.size(); ++i) {
    double v = factd(s->N) / (factd(A[i][0]) * factd(A[i][1]) * factd(A[i][2]) * factd(A[i][3]));
    for (int x = 0; x < 4; ++x) v *= std::pow(std::max(lam[x], 0.0), A[i][x]);
    b[i] = v;
  }
  if (!mass_solve(s->N, b)) return fail(BBW_ERR_ARG, "mass matrix factorisation failed");
  for (double& v : b) v /= s->vol[size_t(found)];
  *elem = found;
  return BBW_OK;
}

// ---------------------------------------------------------------------------
// C ABI

namespace {

// Replace the solver's sources: nelem distinct elements (caller's numbering)
// with coefficient vectors coeffs [nelem][Np] sharing the amplitude series
// amp [nsamples]. Waits for the solver's stream before freeing old buffers.
bbw_status install_sources(bbw_solver* s, int64_t nelem, const int64_t* elems, const double* coeffs,
                           const double* amp, int64_t nsamples) {
  if (nelem < 0 || nsamples < 0) return fail(BBW_ERR_ARG, "negative source count or sample count");
  if ((nelem > 0 && (!elems || !coeffs)) || (nsamples > 0 && !amp)) return fail(BBW_ERR_ARG, "NULL argument");
  if (nelem > s->K) return fail(BBW_ERR_ARG, "more source elements than elements");
  std::vector<char> seen(size_t(s->K), 0);
  std::vector<int64_t> ie(static_cast<size_t>(nelem));
  for (int64_t k = 0; k < nelem; ++k) {
    const int64_t e = elems[k];
    if (e < 0 || e >= s->K) return fail(BBW_ERR_ARG, "source element out of range");
    if (seen[size_t(e)]) return fail(BBW_ERR_ARG, "a source element is listed twice");
    seen[size_t(e)] = 1;
    ie[size_t(k)] = s->slot(e);
  }
  for (int64_t i = 0; i < nelem * s->Np; ++i)
    if (!std::isfinite(coeffs[i])) return fail(BBW_ERR_ARG, "non-finite source coefficient");
  for (int64_t i = 0; i < nsamples; ++i)
    if (!std::isfinite(amp[i])) return fail(BBW_ERR_ARG, "non-finite amplitude sample");
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  for (void** p : {&s->d_src, reinterpret_cast<void**>(&s->d_src_groups), reinterpret_cast<void**>(&s->d_src_slots),
                   reinterpret_cast<void**>(&s->d_src_ser), reinterpret_cast<void**>(&s->d_src_amp)}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  s->nsrc = s->n_src_groups = s->n_amp = 0;
  s->src_elems.clear();
  if (nelem == 0 || nsamples == 0) return BBW_OK;
  std::vector<int64_t> groups;
  std::vector<int32_t> slots;
  bbw::source_groups(ie, s->V, &groups, &slots);
  const size_t nvec = size_t(nelem) * s->Np;
  BBW_CUDA(cudaMalloc(&s->d_src, nvec * s->rsz()));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_src_groups), groups.size() * sizeof(int64_t)));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_src_slots), slots.size() * sizeof(int32_t)));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_src_ser), size_t(nelem) * sizeof(int32_t)));
  BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&s->d_src_amp), size_t(nsamples) * sizeof(double)));
  bbw_status st = upload(s, coeffs, s->d_src, nvec);
  if (st != BBW_OK) return st;
  const std::vector<int32_t> ser(static_cast<size_t>(nelem), 0);
  BBW_CUDA(cudaMemcpy(s->d_src_groups, groups.data(), groups.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaMemcpy(s->d_src_slots, slots.data(), slots.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaMemcpy(s->d_src_ser, ser.data(), ser.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaMemcpy(s->d_src_amp, amp, size_t(nsamples) * sizeof(double), cudaMemcpyHostToDevice));
  BBW_CUDA(cudaStreamSynchronize(s->stream));
  s->nsrc = nelem;
  s->n_src_groups = int64_t(groups.size());
  s->n_amp = nsamples;
  s->src_elems.assign(elems, elems + nelem);
  return BBW_OK;
}

}  // namespace

namespace bbw {

void source_groups(const std::vector<int64_t>& ie, int V, std::vector<int64_t>* groups,
                   std::vector<int32_t>* slots) {
  std::vector<std::pair<int64_t, int32_t>> by(ie.size());
  for (size_t k = 0; k < ie.size(); ++k) by[k] = {ie[k], int32_t(k)};
  std::sort(by.begin(), by.end());
  groups->clear();
  slots->clear();
  for (const auto& [e, k] : by) {
    const int64_t g = e / V;
    if (groups->empty() || groups->back() != g) {
      groups->push_back(g);
      slots->insert(slots->end(), size_t(V), -1);
    }
    (*slots)[(groups->size() - 1) * size_t(V) + size_t(e % V)] = k;
  }
}

}  // namespace bbw

extern "C" {

int bbw_version(void) { return 100; }

const char* bbw_last_error(void) { return g_err.c_str(); }

bbw_status bbw_create(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N, int M,
                      int precision, void* cuda_stream, bbw_solver** out) {
  const std::vector<std::pair<int64_t, int64_t>> all = {{0, K}};
  return bbw::create_solver(nverts, vxyz, K, etov, N, M, precision, cuda_stream, &all, out);
}

}  // extern "C"

bbw_status bbw::create_solver(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N, int M,
                              int precision, void* cuda_stream,
                              const std::vector<std::pair<int64_t, int64_t>>* renumber, bbw_solver** out) {
  if (!out) return fail(BBW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!vxyz || !etov || nverts <= 0 || K <= 0) return fail(BBW_ERR_ARG, "empty mesh or NULL array");
  if (K >= bbw::kMaxElements) return fail(BBW_ERR_ARG, "too many elements (limit 2^26)");
  if (N < 1 || N > bbw::kMaxN) return fail(BBW_ERR_UNSUPPORTED, "N must be in 1..9");
  if (M < 0 || M > bbw::kMaxM) return fail(BBW_ERR_UNSUPPORTED, "M must be in 0..3");
  if (precision != 32 && precision != 64) return fail(BBW_ERR_ARG, "precision must be 32 or 64");
  auto* s = new bbw_solver();
  s->M = M;
  s->prec = precision;
  s->Mp = bbw::np3(M);
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  bbw_status st = setup_mesh(s, nverts, vxyz, K, etov, N);
  if (st != BBW_OK) {
    free_solver(s);
    return st;
  }
  if (renumber && !renumber->empty()) {
    for (const auto& [r0, r1] : *renumber)
      if (r0 < 0 || r1 > K || r0 > r1) {
        free_solver(s);
        return fail(BBW_ERR_ARG, "renumbering range out of bounds");
      }
    st = renumber_elements(s, *renumber);
    if (st != BBW_OK) {
      free_solver(s);
      return st;
    }
  }
  projection_coeffs(N, M, s->cj);
  st = get_tables(N, M, precision, &s->op);
  if (st != BBW_OK) {
    free_solver(s);
    return st;
  }
  int team = 0, gpc = 1;
  s->ops->launch_shape(M, precision == 64, &team, &s->V, &gpc);
  s->G = (K + s->V - 1) / s->V;
  const int64_t tiles = (s->G + gpc - 1) / gpc;
  s->grid_stage = int(std::min<int64_t>(tiles, int64_t(std::max(1, s->op->per_sm_stage)) * num_sms()));

  const size_t rs = s->rsz();
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  const size_t ng = size_t(s->G) * s->V;  // elements including group padding
  bool ok = alloc(&s->q[0], s->nstate_internal() * rs) && alloc(&s->q[1], s->nstate_internal() * rs) &&
            alloc(&s->res, s->nstate_internal() * rs) && alloc(&s->d_c2, ng * s->Mp * rs) &&
            alloc(&s->d_geom, ng * 9 * rs) && alloc(reinterpret_cast<void**>(&s->d_conn), ng * 16) &&
            alloc(reinterpret_cast<void**>(&s->d_status), 16);
  if (!ok) {
    std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(cudaGetLastError());
    free_solver(s);
    return fail(BBW_ERR_CUDA, msg);
  }
  st = precision == 64 ? upload_geometry<double>(s) : upload_geometry<float>(s);
  if (st == BBW_OK) {
    // [G][4][V]; padding elements have walls on all faces
    const int V = s->V;
    std::vector<int32_t> conn(ng * 4, -1);
    for (int64_t e = 0; e < K; ++e)  // internal slot e, caller's element s->user(e)
      for (int f = 0; f < 4; ++f) {
        const size_t i = size_t(s->user(e)) * 4 + f;
        conn[(size_t(e / V) * 4 + f) * V + size_t(e % V)] =
            s->etoe[i] < 0 ? -1
                           : (int32_t(s->slot(s->etoe[i])) << 5) | (int32_t(s->etof[i]) << 3) | int32_t(s->fperm[i]);
      }
    if (cudaMemcpy(s->d_conn, conn.data(), conn.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(BBW_ERR_CUDA, "connectivity upload failed");
  }
  if (st == BBW_OK) {
    std::vector<double> ones(size_t(K) * s->Mp, 1.0);
    st = bbw_set_c2(s, ones.data());
  }
  if (st != BBW_OK) {
    free_solver(s);
    return st;
  }
  *out = s;
  return BBW_OK;
}

extern "C" {

void bbw_destroy(bbw_solver* s) {
  if (s && s->stream) cudaStreamSynchronize(s->stream);
  else if (s) cudaDeviceSynchronize();
  free_solver(s);
}

bbw_status bbw_info(const bbw_solver* s, int64_t* K, int* N, int* M, int* Np, int* Mp, int* precision) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (K) *K = s->K;
  if (N) *N = s->N;
  if (M) *M = s->M;
  if (Np) *Np = s->Np;
  if (Mp) *Mp = s->Mp;
  if (precision) *precision = s->prec;
  return BBW_OK;
}

bbw_status bbw_get_connectivity(const bbw_solver* s, int32_t* etoe, int8_t* etof, int8_t* fperm) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  const size_t n = size_t(s->K) * 4;
  if (etoe) std::memcpy(etoe, s->etoe.data(), n * 4);
  if (etof) std::memcpy(etof, s->etof.data(), n);
  if (fperm) std::memcpy(fperm, s->fperm.data(), n);
  return BBW_OK;
}

bbw_status bbw_get_face_node_map(const bbw_solver* s, int64_t* nmap) {
  if (!s || !nmap) return fail(BBW_ERR_ARG, "NULL argument");
  const int Nfp = s->Nfp;
  std::vector<int> fidx(4 * Nfp), nidx(24 * Nfp);
  s->ops->face_maps(fidx.data(), nidx.data());
  for (int64_t e = 0; e < s->K; ++e)
    for (int f = 0; f < 4; ++f) {
      const size_t slot = size_t(e) * 4 + f;
      for (int a = 0; a < Nfp; ++a) {
        int64_t v = -1;
        if (s->etoe[slot] >= 0)
          v = int64_t(s->etoe[slot]) * s->Np + nidx[(s->etof[slot] * 6 + s->fperm[slot]) * Nfp + a];
        nmap[slot * Nfp + a] = v;
      }
    }
  return BBW_OK;
}

bbw_status bbw_get_geometry(const bbw_solver* s, double* grad, double* vol) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (grad) std::memcpy(grad, s->grad.data(), s->grad.size() * 8);
  if (vol) std::memcpy(vol, s->vol.data(), s->vol.size() * 8);
  return BBW_OK;
}

bbw_status bbw_mesh_analyze(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N,
                            int32_t* etoe, int8_t* etof, int8_t* fperm, int64_t* nmap, double* grad,
                            double* vol) {
  if (!vxyz || !etov || nverts <= 0 || K <= 0) return fail(BBW_ERR_ARG, "empty mesh or NULL array");
  if (K >= bbw::kMaxElements) return fail(BBW_ERR_ARG, "too many elements (limit 2^26)");
  if (N < 1 || N > bbw::kMaxN) return fail(BBW_ERR_UNSUPPORTED, "N must be in 1..9");
  bbw_solver s;
  bbw_status st = setup_mesh(&s, nverts, vxyz, K, etov, N);
  if (st != BBW_OK) return st;
  st = bbw_get_connectivity(&s, etoe, etof, fperm);
  if (st == BBW_OK && nmap) st = bbw_get_face_node_map(&s, nmap);
  if (st == BBW_OK) st = bbw_get_geometry(&s, grad, vol);
  return st;
}

bbw_status bbw_set_c2(bbw_solver* s, const double* c2) {
  if (!s || !c2) return fail(BBW_ERR_ARG, "NULL argument");
  const size_t n = size_t(s->K) * s->Mp;
  for (size_t i = 0; i < n; ++i)
    if (!(c2[i] > 0.0) || !std::isfinite(c2[i]))
      return fail(BBW_ERR_NONPOS_C2, "c^2 coefficient " + std::to_string(i) + " is not positive and finite");
  bbw_status st = upload_grouped(s, c2, s->Mp, 1.0, s->d_c2);
  if (st != BBW_OK) return st;
  s->c2.assign(c2, c2 + n);
  return BBW_OK;
}

bbw_status bbw_set_params(bbw_solver* s, double tau_p, double tau_u) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (!(tau_p >= 0.0) || !(tau_u >= 0.0) || !std::isfinite(tau_p) || !std::isfinite(tau_u))
    return fail(BBW_ERR_ARG, "penalty parameters must be finite and >= 0");
  s->tau_p = tau_p;
  s->tau_u = tau_u;
  return BBW_OK;
}

bbw_status bbw_set_state(bbw_solver* s, const double* q, const double* res, double t) {
  if (!s || !q) return fail(BBW_ERR_ARG, "NULL argument");
  bbw_status st = upload_state(s, q, s->q[s->cur]);
  if (st != BBW_OK) return st;
  if (res) {
    st = upload_state(s, res, s->res);
    if (st != BBW_OK) return st;
  } else {
    BBW_CUDA(cudaMemsetAsync(s->res, 0, s->nstate_internal() * s->rsz(), s->stream));
  }
  s->t = t;
  s->stages = 0;
  s->steps = 0;
  return BBW_OK;
}

bbw_status bbw_set_state_device(bbw_solver* s, const void* q, const void* res, int dtype, double t) {
  if (!s || !q) return fail(BBW_ERR_ARG, "NULL argument");
  if (dtype != 32 && dtype != 64) return fail(BBW_ERR_ARG, "dtype must be 32 or 64");
  BBW_CUDA(bbw::copy_to_internal(q, dtype, s->q[s->cur], s->prec, s->K, s->Np, s->V, s->d_perm, s->stream));
  if (res)
    BBW_CUDA(bbw::copy_to_internal(res, dtype, s->res, s->prec, s->K, s->Np, s->V, s->d_perm, s->stream));
  else
    BBW_CUDA(cudaMemsetAsync(s->res, 0, s->nstate_internal() * s->rsz(), s->stream));
  s->t = t;
  s->stages = 0;
  s->steps = 0;
  return BBW_OK;
}

bbw_status bbw_get_state(bbw_solver* s, double* q, double* res, double* t) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  bbw_status st = check_status(s);
  if (st != BBW_OK) return st;
  if (q) {
    st = download_state(s, s->q[s->cur], q);
    if (st != BBW_OK) return st;
  }
  if (res) {
    st = download_state(s, s->res, res);
    if (st != BBW_OK) return st;
  }
  if (t) *t = s->t;
  return BBW_OK;
}

bbw_status bbw_get_state_device(bbw_solver* s, void* q, void* res, int dtype) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (dtype != 32 && dtype != 64) return fail(BBW_ERR_ARG, "dtype must be 32 or 64");
  if (q) BBW_CUDA(bbw::copy_to_user(s->q[s->cur], s->prec, q, dtype, s->K, s->Np, s->V, s->d_inv, s->stream));
  if (res) BBW_CUDA(bbw::copy_to_user(s->res, s->prec, res, dtype, s->K, s->Np, s->V, s->d_inv, s->stream));
  return BBW_OK;
}

bbw_status bbw_set_source(bbw_solver* s, int64_t elem, const double* coeffs, const double* amp, int64_t nsamples) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (!coeffs) return fail(BBW_ERR_ARG, "NULL argument");
  return install_sources(s, 1, &elem, coeffs, amp, nsamples);
}

bbw_status bbw_set_forcing(bbw_solver* s, int64_t nelem, const int64_t* elems, const double* coeffs,
                           const double* amp, int64_t nsamples) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return install_sources(s, nelem, elems, coeffs, amp, nsamples);
}

bbw_status bbw_set_point_source(bbw_solver* s, const double* xs, const double* amp, int64_t nsamples,
                                int64_t* elem) {
  if (!s || !xs) return fail(BBW_ERR_ARG, "NULL argument");
  int64_t found = -1;
  std::vector<double> b;
  bbw_status st = bbw::point_source_vector(s, xs, 0, s->K, &found, &b);
  if (st != BBW_OK) return st;
  if (elem) *elem = found;
  return install_sources(s, 1, &found, b.data(), amp, nsamples);
}

bbw_status bbw_clear_source(bbw_solver* s) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return install_sources(s, 0, nullptr, nullptr, nullptr, 0);
}

bbw_status bbw_stage(bbw_solver* s, int stage, double dt) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (stage < 0 || stage > 4) return fail(BBW_ERR_ARG, "stage must be in 0..4");
  if (!std::isfinite(dt)) return fail(BBW_ERR_ARG, "dt is not finite");
  return s->prec == 64 ? launch_stage<double>(s, stage, dt) : launch_stage<float>(s, stage, dt);
}

bbw_status bbw_step(bbw_solver* s, double dt, int64_t nsteps) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (nsteps < 0) return fail(BBW_ERR_ARG, "nsteps < 0");
  for (int64_t i = 0; i < nsteps; ++i)
    for (int st = 0; st < 5; ++st) {
      bbw_status r = bbw_stage(s, st, dt);
      if (r != BBW_OK) return r;
    }
  return BBW_OK;
}

bbw_status bbw_cfl_dt(const bbw_solver* s, double cfl, double* dt) {
  if (!s || !dt) return fail(BBW_ERR_ARG, "NULL argument");
  if (!(cfl > 0.0)) return fail(BBW_ERR_ARG, "cfl must be > 0");
  double cmax = 0.0, ratio = 0.0;
  for (double v : s->c2) cmax = std::max(cmax, v);
  for (int64_t e = 0; e < s->K; ++e)
    for (int f = 0; f < 4; ++f) {
      const double* g = &s->grad[size_t(e) * 12 + 3 * f];
      ratio = std::max(ratio, 3.0 * std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
    }
  const double cn = (s->N + 1) * (s->N + 3) / 3.0;
  *dt = cfl / (std::sqrt(cmax) * cn * ratio);
  return BBW_OK;
}

bbw_status bbw_advance(bbw_solver* s, double T, double cfl, double* dt_used, int64_t* nsteps) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (!(T >= 0.0)) return fail(BBW_ERR_ARG, "T must be >= 0");
  double dt = 0.0;
  bbw_status st = bbw_cfl_dt(s, cfl, &dt);
  if (st != BBW_OK) return st;
  const int64_t n = int64_t(std::ceil(T / dt));
  const double h = n > 0 ? T / double(n) : 0.0;
  if (dt_used) *dt_used = h;
  if (nsteps) *nsteps = n;
  return bbw_step(s, h, n);
}

bbw_status bbw_sync(bbw_solver* s) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  return check_status(s);
}

bbw_status bbw_get_time(const bbw_solver* s, double* t, int64_t* stages) {
  if (!s) return fail(BBW_ERR_ARG, "solver is NULL");
  if (t) *t = s->t;
  if (stages) *stages = s->stages;
  return BBW_OK;
}

bbw_status bbw_projection_coeffs(int N, int M, double* c) {
  if (!c) return fail(BBW_ERR_ARG, "c is NULL");
  if (N < 0 || N > bbw::kMaxN || M < 0 || M > 8) return fail(BBW_ERR_ARG, "N or M out of range");
  projection_coeffs(N, M, c);
  return BBW_OK;
}

bbw_status bbw_validate_tables(int N, int M, int precision) {
  if (N < 1 || N > bbw::kMaxN || M < 0 || M > bbw::kMaxM) return fail(BBW_ERR_UNSUPPORTED, "N or M out of range");
  if (precision != 32 && precision != 64) return fail(BBW_ERR_ARG, "precision must be 32 or 64");
  double cj[bbw::kMaxN + 1];
  projection_coeffs(N, M, cj);
  const char* msg = bbw::ops_for(N)->check_tables(M, precision == 64, cj);
  if (msg) return fail(BBW_ERR_ARG, std::string("operator table check failed: ") + msg);
  return BBW_OK;
}

bbw_status bbw_lsrk_coeffs(double* a, double* b, double* c) {
  const auto cs = rk_stage_times();
  for (int i = 0; i < 5; ++i) {
    if (a) a[i] = kRkA[i];
    if (b) b[i] = kRkB[i];
    if (c) c[i] = cs[i];
  }
  return BBW_OK;
}

bbw_status bbw_wadg_update(int N, int M, int precision, int64_t K, const void* rhs, const void* c2, void* out,
                           void* stream) {
  if (N < 1 || N > bbw::kMaxN || M < 0 || M > bbw::kMaxM) return fail(BBW_ERR_UNSUPPORTED, "N or M out of range");
  if (precision != 32 && precision != 64) return fail(BBW_ERR_ARG, "precision must be 32 or 64");
  if (K < 0) return fail(BBW_ERR_ARG, "K < 0");
  if (K == 0) return BBW_OK;
  if (!rhs || !c2 || !out) return fail(BBW_ERR_ARG, "NULL device pointer");
  if (rhs == out) return fail(BBW_ERR_ARG, "out may not alias rhs");
  OpCache* op = nullptr;
  bbw_status st = get_tables(N, M, precision, &op);
  if (st != BBW_OK) return st;
  const bbw::KernelOps* ops = bbw::ops_for(N);
  int team = 0, width = 1, gpc = 1;
  ops->launch_shape(M, precision == 64, &team, &width, &gpc);
  const int64_t per_cta = int64_t(width) * gpc;
  const int64_t tiles = (K + per_cta - 1) / per_cta;
  const int grid = int(std::min<int64_t>(tiles, int64_t(std::max(1, op->per_sm_wadg)) * num_sms()));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == 64) {
    bbw::WadgParams<double> P{static_cast<const double*>(rhs), static_cast<const double*>(c2),
                              static_cast<double*>(out), op->tables, K};
    BBW_CUDA(ops->launch_wadg(M, true, &P, grid, s));
  } else {
    bbw::WadgParams<float> P{static_cast<const float*>(rhs), static_cast<const float*>(c2),
                             static_cast<float*>(out), op->tables, K};
    BBW_CUDA(ops->launch_wadg(M, false, &P, grid, s));
  }
  return BBW_OK;
}

}  // extern "C"
