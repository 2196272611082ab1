// bbw_batch.cu -- many independent BBWADG instances advanced together.
//
// A batch holds n instances (meshes, c^2 fields, states, point sources) of
// uneven size and degree. The instances of one degree N form one bucket: a
// solver over the disjoint union of their meshes, in which every instance
// starts on an element-group boundary (its last group is padded with
// detached unit tetrahedra that stay at rest). The stage kernel is the
// single-mesh one: a disjoint union is just a larger mesh without faces
// between its parts, so one persistent launch per bucket and RK stage covers
// every instance of that degree, and an instance's coefficients are one
// contiguous range of the grouped device arrays.
//
// One RK step over all buckets is captured into a CUDA graph (one fork/join
// branch per bucket, so buckets that do not fill the GPU run side by side)
// and replayed per step. Everything a replay needs lives on the device: the
// step counter (advanced by a one-thread kernel at the end of the step) from
// which the stage kernel picks the sources' amplitude samples, and the source
// tables. Two graphs are kept, one per parity of the ping-pong state buffers
// (a step has five stages, so the parity flips every step); they are
// rebuilt when dt or the penalty parameters change.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "bbw_common.h"
#include "bbw_ops.h"
#include "bbw_solver.h"
#include "bbw_stage.cuh"
#include "bbwadg.h"

using bbw::fail;

namespace {

__global__ void advance_step_kernel(int64_t* step) { step[0] += 1; }

}  // namespace

struct bbw_batch {
  struct Member {
    int bucket = 0;
    int64_t e0 = 0;  // first element in the bucket solver (a multiple of V)
    int64_t K = 0;   // elements of the instance
  };
  struct Bucket {
    int N = 0;
    bbw_solver* s = nullptr;
    std::vector<int> members;            // batch indices, in bucket order
    cudaStream_t side = nullptr;         // branch stream of the step graph
    cudaEvent_t done = nullptr;          // branch join
    int64_t* d_groups = nullptr;         // [members] groups holding a source, ascending
    int32_t* d_slots = nullptr;          // [members][V] source slot per lane of those groups
    int64_t n_groups = 0;
    void* d_vec = nullptr;               // [members][Np] source vectors
    int32_t* d_ser = nullptr;            // [members] amplitude series of member slot x: x
    double* d_amp = nullptr;             // [members][n_amp] amplitude samples, zero padded
    int64_t n_amp = 0;
    std::vector<int64_t> src_elem;       // per member slot: element of its source or -1
    std::vector<std::vector<double>> amp;  // per member slot: its amplitude samples
    int grid0 = 1;                       // persistent grid of the solo solver (CTAs)
    void* d_dtg = nullptr;               // [G] per-group dt (per-instance time steps) or NULL
    int64_t* d_stepsg = nullptr;         // [G] per-group step budget or NULL
  };
  int n = 0, M = 0, prec = 32;
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created here when the caller passed the legacy default stream
  std::vector<Member> members;
  std::vector<Bucket> buckets;
  int64_t* d_step = nullptr;  // device step counter (amplitude sample 5 step + stage)
  double t = 0.0;
  int64_t steps = 0;
  int cur = 0;  // parity of the ping-pong state buffers (equal in all buckets)
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  double graph_dt[2] = {NAN, NAN};
  // launch schedule (bbw_batch_autotune): buckets as concurrent graph
  // branches or one after another, and the persistent grid of every bucket
  // as a fraction of its solo grid
  bool serial = false;
  double grid_factor = 1.0;
  int schedule = 0;
  // per-instance time steps and step budgets (bbw_batch_set_instance_steps;
  // empty: the common dt, no budget) and the instances' own times
  std::vector<double> inst_dt;
  std::vector<int64_t> inst_steps;
  std::vector<double> inst_t;
  bool trial = false;  // autotuner trial steps: per-group dt off (dt = 0)
};

namespace {

void free_batch(bbw_batch* b) {
  if (!b) return;
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto& k : b->buckets) {
    if (k.s) bbw_destroy(k.s);
    if (k.side) cudaStreamDestroy(k.side);
    if (k.done) cudaEventDestroy(k.done);
    for (void* p : {static_cast<void*>(k.d_groups), static_cast<void*>(k.d_slots), k.d_vec,
                    static_cast<void*>(k.d_ser), static_cast<void*>(k.d_amp), k.d_dtg,
                    static_cast<void*>(k.d_stepsg)})
      if (p) cudaFree(p);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_step) cudaFree(b->d_step);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

void invalidate_graphs(bbw_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
    b->graph[p] = nullptr;
    b->graph_dt[p] = NAN;
  }
}

bbw_status check_member(const bbw_batch* b, int i) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (i < 0 || i >= b->n) return fail(BBW_ERR_ARG, "instance index out of range");
  return BBW_OK;
}

// The five stage launches of one bucket on stream st (state parity b->cur).
template <typename real>
bbw_status launch_bucket_step(bbw_batch* b, bbw_batch::Bucket& k, double dt, cudaStream_t st) {
  double a[5], bb[5];
  bbw_lsrk_coeffs(a, bb, nullptr);
  bbw_solver* s = k.s;
  int cur = b->cur;
  for (int stage = 0; stage < 5; ++stage) {
    bbw::StageParams<real> P;
    P.qin = static_cast<const real*>(s->q[cur]);
    P.qout = static_cast<real*>(s->q[1 - cur]);
    P.res = static_cast<real*>(s->res);
    P.c2 = static_cast<const real*>(s->d_c2);
    P.geom = static_cast<const real*>(s->d_geom);
    P.conn = s->d_conn;
    P.tables = s->op->tables;
    P.G = s->G;
    P.a = real(a[stage]);
    P.b = real(bb[stage]);
    P.dt = real(dt);
    P.tau_p = real(s->tau_p);
    P.tau_u = real(s->tau_u);
    P.n_src_groups = k.n_groups;
    P.src_groups = k.d_groups;
    P.src_slots = k.d_slots;
    P.src_vec = static_cast<const real*>(k.d_vec);
    P.src_ser = k.d_ser;
    P.src_amp = k.d_amp;
    P.n_amp = k.n_amp;
    P.step_dev = b->d_step;
    P.step_host = 0;
    P.stage = stage;
    P.status = s->d_status;
    // autotuner trials step with dt = 0 (no per-group dt) but keep the
    // budgets, so that finished instances stay untouched (residual included)
    if (!b->trial) P.dt_group = static_cast<const real*>(k.d_dtg);
    P.steps_group = k.d_stepsg;
    BBW_CUDA(s->ops->launch_stage(s->M, s->prec == 64, &P, s->grid_stage, st));
    cur = 1 - cur;
  }
  return BBW_OK;
}

// One RK step of every bucket, forked onto the bucket streams and joined back
// onto the batch stream, then the device step counter advanced.
bbw_status enqueue_step(bbw_batch* b, double dt) {
  if (b->serial) {
    for (auto& k : b->buckets) {
      bbw_status r = b->prec == 64 ? launch_bucket_step<double>(b, k, dt, b->stream)
                                   : launch_bucket_step<float>(b, k, dt, b->stream);
      if (r != BBW_OK) return r;
    }
  } else {
    BBW_CUDA(cudaEventRecord(b->fork, b->stream));
    for (auto& k : b->buckets) {
      BBW_CUDA(cudaStreamWaitEvent(k.side, b->fork, 0));
      bbw_status r = b->prec == 64 ? launch_bucket_step<double>(b, k, dt, k.side)
                                   : launch_bucket_step<float>(b, k, dt, k.side);
      if (r != BBW_OK) return r;
      BBW_CUDA(cudaEventRecord(k.done, k.side));
      BBW_CUDA(cudaStreamWaitEvent(b->stream, k.done, 0));
    }
  }
  advance_step_kernel<<<1, 1, 0, b->stream>>>(b->d_step);
  BBW_CUDA(cudaGetLastError());
  return BBW_OK;
}

bbw_status build_graph(bbw_batch* b, int parity, double dt) {
  if (b->graph[parity]) cudaGraphExecDestroy(b->graph[parity]);
  b->graph[parity] = nullptr;
  const int saved = b->cur;
  b->cur = parity;
  cudaGraph_t g = nullptr;
  BBW_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  bbw_status r = enqueue_step(b, dt);
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->cur = saved;
  if (r != BBW_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return fail(BBW_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
  const cudaError_t ei = cudaGraphInstantiate(&b->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(BBW_ERR_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(ei));
  b->graph_dt[parity] = dt;
  return BBW_OK;
}

// Member element e (the caller's order, 0 <= e < K) sits at internal slot
// s->slot(e0 + e) - e0 of the member's groups (renumbered within the member).
template <typename T>
void fill_member_state(const bbw_solver* s, const double* src, int64_t e0, int64_t K, T* p) {
  // [G_i][4][Np][V] from [4][K][Np]; padding lanes zero
  const int Np = s->Np, V = s->V;
  const int64_t Gi = (K + V - 1) / V;
  std::memset(p, 0, size_t(Gi) * 4 * Np * V * sizeof(T));
  for (int f = 0; f < 4; ++f)
    for (int64_t e = 0; e < K; ++e) {
      const int64_t ie = s->slot(e0 + e) - e0;
      const double* row = src + (size_t(f) * K + e) * Np;
      for (int i = 0; i < Np; ++i) p[((size_t(ie / V) * 4 + f) * Np + i) * V + size_t(ie % V)] = T(row[i]);
    }
}

template <typename T>
void take_member_state(const bbw_solver* s, const T* p, int64_t e0, int64_t K, double* dst) {
  const int Np = s->Np, V = s->V;
  for (int f = 0; f < 4; ++f)
    for (int64_t e = 0; e < K; ++e) {
      const int64_t ie = s->slot(e0 + e) - e0;
      double* row = dst + (size_t(f) * K + e) * Np;
      for (int i = 0; i < Np; ++i) row[i] = double(p[((size_t(ie / V) * 4 + f) * Np + i) * V + size_t(ie % V)]);
    }
}

// host [4][K_i][Np] -> the member's contiguous range of a grouped device state
bbw_status upload_member_state(bbw_batch* b, int i, const double* src, void* base) {
  const auto& m = b->members[size_t(i)];
  bbw_solver* s = b->buckets[size_t(m.bucket)].s;
  const int64_t Gi = (m.K + s->V - 1) / s->V;
  const size_t n = size_t(Gi) * 4 * s->Np * s->V;
  bbw_status st = bbw::ensure_pinned(s, n * 8);
  if (st != BBW_OK) return st;
  if (s->prec == 64)
    fill_member_state(s, src, m.e0, m.K, static_cast<double*>(s->pinned));
  else
    fill_member_state(s, src, m.e0, m.K, static_cast<float*>(s->pinned));
  char* dst = static_cast<char*>(base) + size_t(m.e0) * 4 * s->Np * s->rsz();
  BBW_CUDA(cudaMemcpyAsync(dst, s->pinned, n * s->rsz(), cudaMemcpyHostToDevice, b->stream));
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  return BBW_OK;
}

bbw_status download_member_state(bbw_batch* b, int i, const void* base, double* dst) {
  const auto& m = b->members[size_t(i)];
  bbw_solver* s = b->buckets[size_t(m.bucket)].s;
  const int64_t Gi = (m.K + s->V - 1) / s->V;
  const size_t n = size_t(Gi) * 4 * s->Np * s->V;
  bbw_status st = bbw::ensure_pinned(s, n * 8);
  if (st != BBW_OK) return st;
  const char* src = static_cast<const char*>(base) + size_t(m.e0) * 4 * s->Np * s->rsz();
  BBW_CUDA(cudaMemcpyAsync(s->pinned, src, n * s->rsz(), cudaMemcpyDeviceToHost, b->stream));
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  if (s->prec == 64)
    take_member_state(s, static_cast<const double*>(s->pinned), m.e0, m.K, dst);
  else
    take_member_state(s, static_cast<const float*>(s->pinned), m.e0, m.K, dst);
  return BBW_OK;
}

// The bucket's source-group list from the members' source elements, and the
// amplitude series of every member slot, zero padded to the longest. The
// number of groups and the series length are kernel parameters, so the step
// graphs are rebuilt.
bbw_status upload_sources(bbw_batch* b, bbw_batch::Bucket& k) {
  std::vector<int64_t> ie;
  std::vector<int32_t> slot_of;  // source index -> member slot
  int64_t namp = 0;
  for (size_t slot = 0; slot < k.src_elem.size(); ++slot) {
    if (k.src_elem[slot] < 0) continue;
    ie.push_back(k.s->slot(k.src_elem[slot]));  // internal position of the source element
    slot_of.push_back(int32_t(slot));
    namp = std::max<int64_t>(namp, int64_t(k.amp[slot].size()));
  }
  std::vector<int64_t> g;
  std::vector<int32_t> sl;
  bbw::source_groups(ie, k.s->V, &g, &sl);
  for (auto& x : sl)
    if (x >= 0) x = slot_of[size_t(x)];  // the kernel indexes vectors and series by member slot
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  if (namp != k.n_amp) {
    if (k.d_amp) cudaFree(k.d_amp);
    k.d_amp = nullptr;
    k.n_amp = 0;
    if (namp > 0) BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&k.d_amp), size_t(namp) * k.amp.size() * sizeof(double)));
    k.n_amp = namp;
  }
  if (namp > 0) {
    std::vector<double> flat(size_t(namp) * k.amp.size(), 0.0);
    for (size_t slot = 0; slot < k.amp.size(); ++slot)
      std::copy(k.amp[slot].begin(), k.amp[slot].end(), flat.begin() + ptrdiff_t(slot * size_t(namp)));
    BBW_CUDA(cudaMemcpy(k.d_amp, flat.data(), flat.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  k.n_groups = namp > 0 ? int64_t(g.size()) : 0;
  if (!g.empty()) {
    BBW_CUDA(cudaMemcpy(k.d_groups, g.data(), g.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    BBW_CUDA(cudaMemcpy(k.d_slots, sl.data(), sl.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  invalidate_graphs(b);
  return BBW_OK;
}

}  // namespace

extern "C" {

bbw_status bbw_batch_create(int n, const int64_t* nverts, const double* const* vxyz, const int64_t* K,
                            const int64_t* const* etov, const int* N, int M, int precision, void* cuda_stream,
                            bbw_batch** out) {
  if (!out) return fail(BBW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !nverts || !vxyz || !K || !etov || !N) return fail(BBW_ERR_ARG, "empty batch or NULL array");
  if (M < 0 || M > bbw::kMaxM) return fail(BBW_ERR_UNSUPPORTED, "M must be in 0..3");
  if (precision != 32 && precision != 64) return fail(BBW_ERR_ARG, "precision must be 32 or 64");
  for (int i = 0; i < n; ++i) {
    if (N[i] < 1 || N[i] > bbw::kMaxN) return fail(BBW_ERR_UNSUPPORTED, "N must be in 1..9");
    if (!vxyz[i] || !etov[i] || nverts[i] <= 0 || K[i] <= 0)
      return fail(BBW_ERR_ARG, "instance " + std::to_string(i) + " has an empty mesh or a NULL array");
  }
  auto* b = new bbw_batch();
  b->n = n;
  b->M = M;
  b->prec = precision;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!b->stream) {  // graphs cannot be captured on the legacy default stream
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(BBW_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  b->members.resize(size_t(n));
  b->inst_t.assign(size_t(n), 0.0);
  std::map<int, std::vector<int>> by_degree;
  for (int i = 0; i < n; ++i) by_degree[N[i]].push_back(i);
  auto bail = [&](bbw_status st) {
    free_batch(b);
    return st;
  };
  for (auto& [deg, ids] : by_degree) {
    bbw_batch::Bucket k;
    k.N = deg;
    k.members = ids;
    int team = 0, V = 1, gpc = 1;
    bbw::ops_for(deg)->launch_shape(M, precision == 64, &team, &V, &gpc);
    // disjoint union, every instance starting on a group boundary
    std::vector<double> xyz;
    std::vector<int64_t> tets;
    int64_t e = 0;
    for (int i : ids) {
      const int64_t vbase = int64_t(xyz.size() / 3);
      xyz.insert(xyz.end(), vxyz[i], vxyz[i] + nverts[i] * 3);
      for (int64_t x = 0; x < K[i] * 4; ++x) {
        if (etov[i][x] < 0 || etov[i][x] >= nverts[i])
          return bail(fail(BBW_ERR_MESH, "instance " + std::to_string(i) + ": vertex id out of range"));
        tets.push_back(vbase + etov[i][x]);
      }
      b->members[size_t(i)] = {int(b->buckets.size()), e, K[i]};
      e += K[i];
      for (; e % V != 0; ++e) {  // detached unit tetrahedron
        const int64_t v0 = int64_t(xyz.size() / 3);
        const double x0 = -2.0 - 2.0 * double(e % 64);
        const double pts[12] = {x0, 0, 0, x0 + 1, 0, 0, x0, 1, 0, x0, 0, 1};
        xyz.insert(xyz.end(), pts, pts + 12);
        for (int c = 0; c < 4; ++c) tets.push_back(v0 + c);
      }
    }
    if (e >= bbw::kMaxElements) return bail(fail(BBW_ERR_ARG, "too many elements of one degree (limit 2^26)"));
    // elements are renumbered for locality within each instance only, so that
    // every instance stays one contiguous range of groups
    std::vector<std::pair<int64_t, int64_t>> ranges;
    for (int i : ids) ranges.emplace_back(b->members[size_t(i)].e0, b->members[size_t(i)].e0 + K[i]);
    bbw_status st = bbw::create_solver(int64_t(xyz.size() / 3), xyz.data(), e, tets.data(), deg, M, precision,
                                       b->stream, &ranges, &k.s);
    if (st != BBW_OK) return bail(st);
    k.src_elem.assign(ids.size(), -1);
    k.amp.assign(ids.size(), std::vector<double>());
    k.grid0 = k.s->grid_stage;
    bool ok = cudaStreamCreateWithFlags(&k.side, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming) == cudaSuccess &&
                    cudaMalloc(reinterpret_cast<void**>(&k.d_groups), ids.size() * sizeof(int64_t)) == cudaSuccess &&
                    cudaMalloc(reinterpret_cast<void**>(&k.d_slots), ids.size() * V * sizeof(int32_t)) == cudaSuccess &&
                    cudaMalloc(&k.d_vec, ids.size() * k.s->Np * k.s->rsz()) == cudaSuccess &&
                    cudaMalloc(reinterpret_cast<void**>(&k.d_ser), ids.size() * sizeof(int32_t)) == cudaSuccess;
    if (ok) {
      std::vector<int32_t> ser(ids.size());
      for (size_t x = 0; x < ser.size(); ++x) ser[x] = int32_t(x);
      ok = cudaMemcpy(k.d_ser, ser.data(), ser.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    b->buckets.push_back(k);
    if (!ok) return bail(fail(BBW_ERR_CUDA, "batch allocation failed"));
    st = upload_sources(b, b->buckets.back());
    if (st != BBW_OK) return bail(st);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b->d_step), sizeof(int64_t)) != cudaSuccess ||
      cudaMemset(b->d_step, 0, sizeof(int64_t)) != cudaSuccess)
    return bail(fail(BBW_ERR_CUDA, "batch allocation failed"));
  *out = b;
  return BBW_OK;
}

void bbw_batch_destroy(bbw_batch* b) {
  if (!b) return;
  if (b->stream)
    cudaStreamSynchronize(b->stream);
  else
    cudaDeviceSynchronize();
  free_batch(b);
}

bbw_status bbw_batch_info(const bbw_batch* b, int* n, int* nbuckets, int64_t* elements) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (n) *n = b->n;
  if (nbuckets) *nbuckets = int(b->buckets.size());
  if (elements) {
    int64_t total = 0;
    for (const auto& k : b->buckets) total += k.s->K;
    *elements = total;
  }
  return BBW_OK;
}

bbw_status bbw_batch_member(const bbw_batch* b, int i, int* N, int64_t* K, int* Np, int* bucket, int64_t* first) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  const auto& m = b->members[size_t(i)];
  const auto& k = b->buckets[size_t(m.bucket)];
  if (N) *N = k.N;
  if (K) *K = m.K;
  if (Np) *Np = k.s->Np;
  if (bucket) *bucket = m.bucket;
  if (first) *first = m.e0;
  return BBW_OK;
}

bbw_status bbw_batch_set_c2(bbw_batch* b, int i, const double* c2) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  if (!c2) return fail(BBW_ERR_ARG, "NULL argument");
  const auto& m = b->members[size_t(i)];
  bbw_solver* s = b->buckets[size_t(m.bucket)].s;
  const int Mp = s->Mp, V = s->V;
  for (int64_t x = 0; x < m.K * Mp; ++x)
    if (!(c2[x] > 0.0) || !std::isfinite(c2[x]))
      return fail(BBW_ERR_NONPOS_C2, "c^2 coefficient " + std::to_string(x) + " is not positive and finite");
  std::copy(c2, c2 + m.K * Mp, s->c2.begin() + m.e0 * Mp);
  // the member's groups of the [G][Mp][V] array; padding lanes keep c^2 = 1
  const int64_t Gi = (m.K + V - 1) / V;
  const size_t cnt = size_t(Gi) * Mp * V;
  st = bbw::ensure_pinned(s, cnt * 8);
  if (st != BBW_OK) return st;
  auto fill = [&](auto* p) {
    using T = std::remove_pointer_t<decltype(p)>;
    for (int64_t e = 0; e < Gi * V; ++e)
      for (int w = 0; w < Mp; ++w)
        p[(size_t(e / V) * Mp + w) * V + size_t(e % V)] =
            T(e < m.K ? c2[size_t(s->user(m.e0 + e) - m.e0) * Mp + w] : 1.0);
  };
  if (s->prec == 64)
    fill(static_cast<double*>(s->pinned));
  else
    fill(static_cast<float*>(s->pinned));
  char* dst = static_cast<char*>(s->d_c2) + size_t(m.e0) * Mp * s->rsz();
  BBW_CUDA(cudaMemcpyAsync(dst, s->pinned, cnt * s->rsz(), cudaMemcpyHostToDevice, b->stream));
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  return BBW_OK;
}

bbw_status bbw_batch_set_params(bbw_batch* b, double tau_p, double tau_u) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  for (auto& k : b->buckets) {
    bbw_status st = bbw_set_params(k.s, tau_p, tau_u);
    if (st != BBW_OK) return st;
  }
  invalidate_graphs(b);
  return BBW_OK;
}

bbw_status bbw_batch_set_state(bbw_batch* b, int i, const double* q, const double* res) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  if (!q) return fail(BBW_ERR_ARG, "NULL argument");
  bbw_solver* s = b->buckets[size_t(b->members[size_t(i)].bucket)].s;
  st = upload_member_state(b, i, q, s->q[b->cur]);
  if (st != BBW_OK) return st;
  if (res) return upload_member_state(b, i, res, s->res);
  std::vector<double> zero(size_t(4) * b->members[size_t(i)].K * s->Np, 0.0);
  return upload_member_state(b, i, zero.data(), s->res);
}

bbw_status bbw_batch_get_state(bbw_batch* b, int i, double* q, double* res) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  for (auto& k : b->buckets) {
    st = bbw::check_status(k.s);
    if (st != BBW_OK) return st;
  }
  bbw_solver* s = b->buckets[size_t(b->members[size_t(i)].bucket)].s;
  if (q) {
    st = download_member_state(b, i, s->q[b->cur], q);
    if (st != BBW_OK) return st;
  }
  if (res) return download_member_state(b, i, s->res, res);
  return BBW_OK;
}

bbw_status bbw_batch_set_point_source(bbw_batch* b, int i, const double* xs, const double* amp, int64_t nsamples,
                                      int64_t* elem) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  if (!xs || (nsamples > 0 && !amp)) return fail(BBW_ERR_ARG, "NULL argument");
  if (nsamples < 0) return fail(BBW_ERR_ARG, "nsamples < 0");
  for (int64_t x = 0; x < nsamples; ++x)
    if (!std::isfinite(amp[x])) return fail(BBW_ERR_ARG, "non-finite amplitude sample");
  const auto& m = b->members[size_t(i)];
  auto& k = b->buckets[size_t(m.bucket)];
  bbw_solver* s = k.s;
  int64_t found = -1;
  std::vector<double> vec;
  st = bbw::point_source_vector(s, xs, m.e0, m.e0 + m.K, &found, &vec);
  if (st != BBW_OK) return st;
  const int slot = int(std::find(k.members.begin(), k.members.end(), i) - k.members.begin());
  k.src_elem[size_t(slot)] = found;
  k.amp[size_t(slot)].assign(amp, amp + nsamples);
  std::vector<float> vf(vec.begin(), vec.end());
  const void* vsrc = s->prec == 64 ? static_cast<const void*>(vec.data()) : static_cast<const void*>(vf.data());
  BBW_CUDA(cudaMemcpyAsync(static_cast<char*>(k.d_vec) + size_t(slot) * s->Np * s->rsz(), vsrc, s->Np * s->rsz(),
                           cudaMemcpyHostToDevice, b->stream));
  st = upload_sources(b, k);
  if (st != BBW_OK) return st;
  if (elem) *elem = found - m.e0;
  return BBW_OK;
}

bbw_status bbw_batch_clear_sources(bbw_batch* b) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  for (auto& k : b->buckets) {
    std::fill(k.src_elem.begin(), k.src_elem.end(), -1);
    for (auto& a : k.amp) a.clear();
    bbw_status st = upload_sources(b, k);
    if (st != BBW_OK) return st;
  }
  return BBW_OK;
}

bbw_status bbw_batch_member_cfl_dt(const bbw_batch* b, int i, double cfl, double* dt) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  if (!dt) return fail(BBW_ERR_ARG, "NULL argument");
  if (!(cfl > 0.0)) return fail(BBW_ERR_ARG, "cfl must be > 0");
  double best = INFINITY;
  {
    const auto& m = b->members[size_t(i)];
    const bbw_solver* s = b->buckets[size_t(m.bucket)].s;
    double cmax = 0.0, ratio = 0.0;
    for (int64_t x = m.e0 * s->Mp; x < (m.e0 + m.K) * s->Mp; ++x) cmax = std::max(cmax, s->c2[size_t(x)]);
    for (int64_t e = m.e0; e < m.e0 + m.K; ++e)
      for (int f = 0; f < 4; ++f) {
        const double* g = &s->grad[size_t(e) * 12 + 3 * f];
        ratio = std::max(ratio, 3.0 * std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
      }
    const double cn = (s->N + 1) * (s->N + 3) / 3.0;
    best = std::min(best, cfl / (std::sqrt(cmax) * cn * ratio));
  }
  *dt = best;
  return BBW_OK;
}

bbw_status bbw_batch_cfl_dt(const bbw_batch* b, double cfl, double* dt) {
  if (!b || !dt) return fail(BBW_ERR_ARG, "NULL argument");
  if (!(cfl > 0.0)) return fail(BBW_ERR_ARG, "cfl must be > 0");
  double best = INFINITY;
  for (int i = 0; i < b->n; ++i) {
    double d = 0.0;
    bbw_status st = bbw_batch_member_cfl_dt(b, i, cfl, &d);
    if (st != BBW_OK) return st;
    best = std::min(best, d);
  }
  *dt = best;
  return BBW_OK;
}

bbw_status bbw_batch_set_instance_steps(bbw_batch* b, const double* dt, const int64_t* nsteps) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  for (int i = 0; i < b->n; ++i) {
    if (dt && !(std::isfinite(dt[i]) && dt[i] >= 0.0)) return fail(BBW_ERR_ARG, "instance dt must be finite and >= 0");
    if (nsteps && nsteps[i] < 0) return fail(BBW_ERR_ARG, "instance step budget must be >= 0");
  }
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  if (dt)
    b->inst_dt.assign(dt, dt + b->n);
  else
    b->inst_dt.clear();
  if (nsteps)
    b->inst_steps.assign(nsteps, nsteps + b->n);
  else
    b->inst_steps.clear();
  for (auto& k : b->buckets) {
    bbw_solver* s = k.s;
    const size_t esz = b->prec == 64 ? sizeof(double) : sizeof(float);
    if (k.d_dtg) cudaFree(k.d_dtg);
    if (k.d_stepsg) cudaFree(k.d_stepsg);
    k.d_dtg = nullptr;
    k.d_stepsg = nullptr;
    // groups of no member (none exist: members tile the bucket) stay inert: dt 0, budget 0
    std::vector<double> gdt(size_t(s->G), 0.0);
    std::vector<int64_t> gst(size_t(s->G), 0);
    for (int i : k.members) {
      const auto& m = b->members[size_t(i)];
      for (int64_t g = m.e0 / s->V; g < (m.e0 + m.K + s->V - 1) / s->V; ++g) {
        if (dt) gdt[size_t(g)] = dt[i];
        if (nsteps) gst[size_t(g)] = nsteps[i];
      }
    }
    if (dt) {
      BBW_CUDA(cudaMalloc(&k.d_dtg, size_t(s->G) * esz));
      if (b->prec == 64) {
        BBW_CUDA(cudaMemcpy(k.d_dtg, gdt.data(), gdt.size() * esz, cudaMemcpyHostToDevice));
      } else {
        std::vector<float> f(gdt.begin(), gdt.end());
        BBW_CUDA(cudaMemcpy(k.d_dtg, f.data(), f.size() * esz, cudaMemcpyHostToDevice));
      }
    }
    if (nsteps) {
      BBW_CUDA(cudaMalloc(reinterpret_cast<void**>(&k.d_stepsg), size_t(s->G) * sizeof(int64_t)));
      BBW_CUDA(cudaMemcpy(k.d_stepsg, gst.data(), gst.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
  }
  invalidate_graphs(b);
  return BBW_OK;
}

bbw_status bbw_batch_instance_time(const bbw_batch* b, int i, double* t, int64_t* steps) {
  bbw_status st = check_member(b, i);
  if (st != BBW_OK) return st;
  if (t) *t = b->inst_t[size_t(i)];
  if (steps)
    *steps = b->inst_steps.empty() ? b->steps : std::min(b->steps, b->inst_steps[size_t(i)]);
  return BBW_OK;
}

bbw_status bbw_batch_step(bbw_batch* b, double dt, int64_t nsteps, int use_graph) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (nsteps < 0) return fail(BBW_ERR_ARG, "nsteps < 0");
  if (!std::isfinite(dt)) return fail(BBW_ERR_ARG, "dt is not finite");
  for (int64_t x = 0; x < nsteps; ++x) {
    if (use_graph) {
      const int p = b->cur;
      if (!b->graph[p] || b->graph_dt[p] != dt) {
        bbw_status st = build_graph(b, p, dt);
        if (st != BBW_OK) return st;
      }
      BBW_CUDA(cudaGraphLaunch(b->graph[p], b->stream));
    } else {
      bbw_status st = enqueue_step(b, dt);
      if (st != BBW_OK) return st;
    }
    b->cur = 1 - b->cur;
    for (auto& k : b->buckets) {
      k.s->cur = b->cur;
      k.s->stages += 5;
      k.s->t += dt;
    }
    if (!b->trial)
      for (int i = 0; i < b->n; ++i)
        if (b->inst_steps.empty() || b->steps < b->inst_steps[size_t(i)])
          b->inst_t[size_t(i)] += b->inst_dt.empty() ? dt : b->inst_dt[size_t(i)];
    b->t += dt;
    b->steps += 1;
  }
  return BBW_OK;
}

bbw_status bbw_batch_autotune(bbw_batch* b, int steps, int* schedule, double* ms_per_step) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (steps < 1) return fail(BBW_ERR_ARG, "steps must be >= 1");
  // candidate schedules: (serial, grid factor); 0 is the default
  static const struct {
    bool serial;
    double factor;
  } cand[] = {{false, 1.0}, {true, 1.0}, {false, 0.5}, {false, 2.0}};
  constexpr int ncand = int(sizeof(cand) / sizeof(cand[0]));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BBW_CUDA(cudaEventCreate(&e0));
  BBW_CUDA(cudaEventCreate(&e1));
  auto apply = [&](int c) {
    b->serial = cand[c].serial;
    b->grid_factor = cand[c].factor;
    b->schedule = c;
    for (auto& k : b->buckets) k.s->grid_stage = std::max(1, int(std::lround(k.grid0 * cand[c].factor)));
    invalidate_graphs(b);
  };
  // trial steps have dt = 0: stage 0 sets res = 0 (a_0 = 0) and every stage
  // then writes q_out = q_in + b * 0, so the state and the time stay as they
  // are while the kernels do their full work
  const double saved_t = b->t;
  const int64_t saved_steps = b->steps;
  b->trial = true;
  float best = INFINITY;
  int best_c = 0;
  bbw_status st = BBW_OK;
  for (int c = 0; c < ncand && st == BBW_OK; ++c) {
    apply(c);
    st = bbw_batch_step(b, 0.0, 2, 1);  // build both parities' graphs, warm up
    if (st != BBW_OK) break;
    if (cudaEventRecord(e0, b->stream) != cudaSuccess) st = fail(BBW_ERR_CUDA, "event record failed");
    if (st == BBW_OK) st = bbw_batch_step(b, 0.0, steps, 1);
    if (st == BBW_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) st = fail(BBW_ERR_CUDA, "event record failed");
    if (st == BBW_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(BBW_ERR_CUDA, "event wait failed");
    float ms = 0.f;
    if (st == BBW_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = fail(BBW_ERR_CUDA, "event timing failed");
    if (st == BBW_OK && ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->trial = false;
  apply(st == BBW_OK ? best_c : 0);
  b->t = saved_t;
  b->steps = saved_steps;
  for (auto& k : b->buckets) k.s->t = saved_t;
  cudaError_t ec = cudaStreamSynchronize(b->stream);
  if (ec == cudaSuccess) ec = cudaMemcpy(b->d_step, &saved_steps, sizeof(int64_t), cudaMemcpyHostToDevice);
  if (st == BBW_OK && ec != cudaSuccess) st = fail(BBW_ERR_CUDA, "step counter restore failed");
  if (st != BBW_OK) return st;
  if (schedule) *schedule = best_c;
  if (ms_per_step) *ms_per_step = double(best) / steps;
  return bbw_batch_sync(b);
}

bbw_status bbw_batch_sync(bbw_batch* b) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  for (auto& k : b->buckets) {
    bbw_status st = bbw::check_status(k.s);
    if (st != BBW_OK) return st;
  }
  return BBW_OK;
}

bbw_status bbw_batch_set_time(bbw_batch* b, double t) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (!std::isfinite(t)) return fail(BBW_ERR_ARG, "t is not finite");
  const int64_t zero = 0;
  BBW_CUDA(cudaStreamSynchronize(b->stream));
  BBW_CUDA(cudaMemcpy(b->d_step, &zero, sizeof(int64_t), cudaMemcpyHostToDevice));
  b->t = t;
  b->steps = 0;
  std::fill(b->inst_t.begin(), b->inst_t.end(), t);
  for (auto& k : b->buckets) {
    k.s->t = t;
    k.s->stages = 0;
  }
  return BBW_OK;
}

bbw_status bbw_batch_get_time(const bbw_batch* b, double* t, int64_t* steps) {
  if (!b) return fail(BBW_ERR_ARG, "batch is NULL");
  if (t) *t = b->t;
  if (steps) *steps = b->steps;
  return BBW_OK;
}

}  // extern "C"
