// bbw_solver.h -- internal to libbbwadg: the solver object and the host
// helpers shared by the translation units of the C ABI (bbw_api.cu,
// bbw_batch.cu). Not installed; callers see only include/bbwadg.h.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "bbw_common.h"
#include "bbw_ops.h"
#include "bbwadg.h"

namespace bbw {

// per-process cache of device tables and launch grids for the stateless
// operator entry point (keyed by device, N, M, precision)
struct OpCache {
  void* tables = nullptr;
  int per_sm_stage = 0, per_sm_wadg = 0;
};

// Record msg as the thread's last error and return s.
inline bbw_status fail(bbw_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define BBW_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bbw::fail(BBW_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace bbw

struct AdjointData;  // bbw_adjoint.cu

struct bbw_solver {
  int N = 0, M = 0, prec = 32;
  int64_t K = 0;
  int Np = 0, Nfp = 0, Mp = 0;
  cudaStream_t stream = nullptr;
  const bbw::KernelOps* ops = nullptr;
  bbw::OpCache* op = nullptr;
  int grid_stage = 1;
  std::vector<double> vxyz;
  std::vector<int64_t> etov;
  std::vector<double> grad;  // [K][4][3]
  std::vector<double> vol;   // [K]
  std::vector<int32_t> etoe;
  std::vector<int8_t> etof, fperm;
  std::vector<double> c2;  // [K][Mp]
  double cj[bbw::kMaxN + 1] = {};
  void* q[2] = {nullptr, nullptr};
  void* res = nullptr;
  void* d_c2 = nullptr;
  void* d_geom = nullptr;
  int32_t* d_conn = nullptr;
  // sources (bbw_set_source / bbw_set_forcing): the source elements' groups
  // in ascending order, the source index of each element lane of a listed
  // group (-1: none), the source vectors and their one amplitude series
  void* d_src = nullptr;            // [nsrc][Np] source vectors
  int64_t* d_src_groups = nullptr;  // [n_src_groups]
  int32_t* d_src_slots = nullptr;   // [n_src_groups][V]
  int32_t* d_src_ser = nullptr;     // [nsrc] amplitude series of each source (all 0)
  double* d_src_amp = nullptr;      // [n_amp] amplitude samples
  int64_t nsrc = 0, n_src_groups = 0, n_amp = 0;
  std::vector<int64_t> src_elems;   // the caller's element of each source
  unsigned int* d_status = nullptr;
  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  void* d_stage = nullptr;  // FP64 user-layout staging of host state transfers
  size_t d_stage_bytes = 0;
  int cur = 0;
  double t = 0.0;
  int64_t stages = 0;
  int64_t steps = 0;  // completed RK steps since the last set_state: amplitude sample 5 steps + stage
  double tau_p = 1.0, tau_u = 1.0;
  AdjointData* adj = nullptr;  // receivers, recorded run, adjoint buffers (bbw_adjoint.cu)
  void* vout = nullptr;        // if set, the next stage also stores its pressure bracket there (bbw_record)
  // element renumbering for locality: internal slot e holds the caller's
  // element perm[e], inv[perm[e]] = e (empty / NULL: the identity)
  std::vector<int32_t> perm, inv;
  int32_t* d_perm = nullptr;
  int32_t* d_inv = nullptr;
  int64_t slot(int64_t e) const { return inv.empty() ? e : inv[size_t(e)]; }    // caller -> internal
  int64_t user(int64_t e) const { return perm.empty() ? e : perm[size_t(e)]; }  // internal -> caller
  int V = 1;        // elements per group of the kernel's layout
  int64_t G = 0;   // number of groups, ceil(K / V)
  size_t rsz() const { return prec == 64 ? 8 : 4; }
  size_t nstate() const { return size_t(4) * size_t(K) * size_t(Np); }           // user layout
  size_t nstate_internal() const { return size_t(4) * size_t(G) * V * Np; }      // grouped layout
};

namespace bbw {

// State layout conversions on the device: the ABI's [4][K][Np] ("user")
// and the kernels' grouped [G][4][Np][V] ("internal"), each in FP32 or FP64
// (prec 32 | 64); padding entries of the internal layout are set to zero.
// Internal slot e holds the caller's element perm[e]; inv is the inverse
// (NULL: the identity).
cudaError_t copy_to_internal(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np, int V,
                             const int32_t* perm, cudaStream_t s);
cudaError_t copy_to_user(const void* src, int src_prec, void* dst, int dst_prec, int64_t K, int Np, int V,
                         const int32_t* inv, cudaStream_t s);
// Create a solver (as bbw_create). renumber: element ranges [lo, hi) within
// which the elements are ordered internally by the Morton key of their
// centroids (each range over its own bounding box); NULL or empty: keep the
// caller's order.
bbw_status create_solver(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N, int M,
                         int precision, void* cuda_stream, const std::vector<std::pair<int64_t, int64_t>>* renumber,
                         bbw_solver** out);
// n!, the degree-n multi-indices (alpha_0..alpha_3) in the library order, and
// a solve with the normalised degree-n Bernstein mass matrix (in place;
// false if the factorisation fails).
double factorial(int n);
std::vector<std::array<int, 4>> lattice(int n);
bool solve_mass(int n, std::vector<double>& b);
// Release the adjoint data of a solver (bbw_adjoint.cu); no-op without any.
void free_adjoint(bbw_solver* s);
// Grow the solver's pinned staging buffer to at least bytes.
bbw_status ensure_pinned(bbw_solver* s, size_t bytes);
// Wait for the solver's stream and surface the device status word.
bbw_status check_status(bbw_solver* s);
// Source tables of the stage kernel for a list of source elements (internal
// slots ie[k], k = source index): the ascending list of their groups and, per
// listed group, the source index of each of its V element lanes (-1: none).
void source_groups(const std::vector<int64_t>& ie, int V, std::vector<int64_t>* groups,
                   std::vector<int32_t>* slots);
// Point source at xs searched among elements [e_begin, e_end) (lowest index
// wins on shared faces): its element and the vector M^{-1} B(x_s) / |D| of
// N_p Bernstein coefficients.
bbw_status point_source_vector(const bbw_solver* s, const double* xs, int64_t e_begin, int64_t e_end,
                               int64_t* elem, std::vector<double>* vec);

// Source fields of a stage launch of solver s at stage `stage` of step `step`
// (sources off when on == false).
template <typename P_t, typename real>
void set_stage_sources(const bbw_solver* s, P_t& P, int64_t step, int stage, bool on) {
  P.n_src_groups = on ? s->n_src_groups : 0;
  P.src_groups = s->d_src_groups;
  P.src_slots = s->d_src_slots;
  P.src_vec = static_cast<const real*>(s->d_src);
  P.src_ser = s->d_src_ser;
  P.src_amp = s->d_src_amp;
  P.n_amp = s->n_amp;
  P.step_dev = nullptr;
  P.step_host = step;
  P.stage = stage;
}

}  // namespace bbw
