/*
 * bbwadg.h -- C ABI of the GB300 BBWADG acoustic solver (libbbwadg.so).
 *
 * Bernstein-Bezier weight-adjusted DG (Guo & Chan) for the first-order
 * acoustic wave equation (Eq. 1)
 *
 *     (1/c^2) dp/dt + div u = f,      du/dt + grad p = 0,
 *
 * on affine tetrahedra (Sec. 2), in the strong DG form with penalty fluxes of
 * Eq. (2) and the weight-adjusted mass of Eq. (4). One call of bbw_stage() is
 * one stage of the five-stage low-storage RK4 (Sec. 6.3.1) over all
 * elements, fused in one GPU kernel: sparse Bernstein derivative (Sec. 4),
 * face flux and factored lift L^f = E_L L0 (Sec. 4), the product with the
 * degree-M Bernstein polynomial c^2_M (Eq. 11) and the L2 projection back to
 * degree N by the telescoped form of Eq. (20), and the LSRK update.
 *
 * Conventions
 * -----------
 *  - Barycentrics (Sec. 2): lambda_0 is attached to the element's first vertex
 *    etov[e][0], lambda_m to etov[e][m]. Face f of an element is the face
 *    opposite vertex f ({lambda_f = 0}).
 *  - Multi-index order for degree n (N_p = (n+1)(n+2)(n+3)/6 entries):
 *        for l in 0..n, for k in 0..n-l, for j in 0..n-l-k:
 *            alpha = (n-j-k-l, j, k, l)
 *    Coefficient i of an element is the Bernstein coefficient of
 *    B^n_alpha = n!/(alpha!) lambda^alpha for the i-th alpha in that order.
 *  - State arrays are [4][K][N_p], fields (p, u, v, w), row-major.
 *  - c^2 arrays are [K][M_p], Bernstein coefficients of degree M in the same
 *    order; every coefficient must be > 0 (then c^2_M > 0 everywhere).
 *  - Walls (faces without a neighbour) are p = 0 mirrors: p+ = -p, u+ = u.
 *  - Face orientation code fperm in 0..5: the local vertices of a face are its
 *    three element vertices other than f, in increasing order (v0, v1, v2);
 *    the neighbour's face f' has (w0, w1, w2) likewise. Code c means that
 *    v_x and w_{PERM[c][x]} are the same mesh vertex, with
 *    PERM = {012, 021, 102, 120, 201, 210}.
 *
 * Ownership and errors
 * --------------------
 *  - The caller owns every host array passed in; the library copies what it
 *    needs before returning and keeps no pointer to it.
 *  - The library owns all device buffers of a solver. The *_device calls copy
 *    from/to caller-owned device memory on the solver's stream.
 *  - Every call returns a bbw_status; no exception or abort crosses the ABI.
 *    bbw_last_error() returns a thread-local message for the last failure.
 *  - GPU work is asynchronous on the solver's stream. Asynchronous failures
 *    (a CUDA error, a non-finite value found by the stage kernel) are
 *    reported by the next bbw_sync() or bbw_get_*() call.
 *  - A solver must not be used from two host threads at once.
 */
#ifndef BBWADG_H
#define BBWADG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bbw_solver bbw_solver; /* opaque, library-owned */
typedef struct bbw_batch bbw_batch;   /* opaque, library-owned */
typedef struct bbw_elastic bbw_elastic; /* opaque, library-owned */

typedef enum bbw_status {
  BBW_OK = 0,
  BBW_ERR_ARG = -1,          /* bad argument (null pointer, size, range)       */
  BBW_ERR_MESH = -2,         /* inverted, degenerate or non-manifold mesh      */
  BBW_ERR_NONPOS_C2 = -3,    /* a c^2 Bernstein coefficient is <= 0 or not finite */
  BBW_ERR_CUDA = -4,         /* a CUDA runtime call failed                      */
  BBW_ERR_NONFINITE = -5,    /* the stage kernel produced a NaN or Inf          */
  BBW_ERR_TIMEOUT = -6,      /* reserved for bounded device waits               */
  BBW_ERR_UNSUPPORTED = -7   /* (N, M, precision) not compiled into the library */
} bbw_status;

enum { BBW_MAX_N = 9, BBW_MAX_M = 3 };
enum { BBW_F32 = 32, BBW_F64 = 64 };

/* Library version (major*10000 + minor*100 + patch). */
int bbw_version(void);

/* Thread-local text of the last error; never NULL. */
const char* bbw_last_error(void);

/*
 * Create a solver on the current CUDA device.
 *   vxyz      [nverts][3] vertex coordinates.
 *   etov      [K][4] vertex ids per element (0-based); elements must have
 *             positive orientation (det[v1-v0, v2-v0, v3-v0] > 0).
 *   N         solution degree, 1..BBW_MAX_N.
 *   M         degree of the c^2 approximation, 0..BBW_MAX_M (Sec. 5).
 *   precision BBW_F32 or BBW_F64: arithmetic and storage type on the GPU.
 *   cuda_stream  cudaStream_t to run on (NULL = the legacy default stream).
 * Builds connectivity (faces matched by their vertex triples), geometric
 * factors, operator tables and the projection constants c_j of Theorem 5.3;
 * c^2 starts at 1, the state at 0, tau_p = tau_u = 1, t = 0, no source.
 * Errors: BBW_ERR_ARG, BBW_ERR_MESH (inverted/degenerate element, a face
 * shared by more than two elements), BBW_ERR_UNSUPPORTED, BBW_ERR_CUDA.
 */
bbw_status bbw_create(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov,
                      int N, int M, int precision, void* cuda_stream, bbw_solver** out);

/* Free all device and host memory of a solver (NULL is ignored). */
void bbw_destroy(bbw_solver* s);

/* Sizes of a solver; any output pointer may be NULL. */
bbw_status bbw_info(const bbw_solver* s, int64_t* K, int* N, int* M, int* Np, int* Mp,
                    int* precision);

/*
 * Connectivity (Sec. 4: node-to-node maps on shared faces).
 *   etoe  [K][4] neighbour element across face f, -1 on a wall.
 *   etof  [K][4] the neighbour's local face, -1 on a wall.
 *   fperm [K][4] face orientation code (see Conventions), -1 on a wall.
 */
bbw_status bbw_get_connectivity(const bbw_solver* s, int32_t* etoe, int8_t* etof, int8_t* fperm);

/*
 * Neighbour coefficient of every face node: nmap[e][f][a] is
 * nb * N_p + i, the flat index of the neighbour coefficient that shares the
 * physical domain point of face node a of face f (face nodes enumerated as
 * (b0, b1, b2) over the face's local vertices, b2 outer, b1 inner); -1 on a wall.
 * nmap has K * 4 * (N+1)(N+2)/2 entries.
 */
bbw_status bbw_get_face_node_map(const bbw_solver* s, int64_t* nmap);

/*
 * Host-only mesh analysis, without a GPU or a solver: the same connectivity,
 * face-node map and geometry a solver of degree N builds at bbw_create.
 * Outputs as for bbw_get_connectivity / bbw_get_face_node_map /
 * bbw_get_geometry; nmap, grad and vol may be NULL. Errors: BBW_ERR_ARG,
 * BBW_ERR_MESH, BBW_ERR_UNSUPPORTED (N out of range).
 */
bbw_status bbw_mesh_analyze(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N,
                            int32_t* etoe, int8_t* etof, int8_t* fperm, int64_t* nmap, double* grad,
                            double* vol);

/* Geometry: grad [K][4][3] = d lambda_m / d x_i, vol [K] element volumes. */
bbw_status bbw_get_geometry(const bbw_solver* s, double* grad, double* vol);

/*
 * Per-element Bernstein coefficients of c^2_M (Sec. 5, preprocessing), [K][M_p].
 * Errors: BBW_ERR_NONPOS_C2 if any coefficient is <= 0 or not finite
 * (positivity of the coefficients guarantees c^2_M > 0 by the convex hull
 * property); the solver keeps its previous c^2 then.
 */
bbw_status bbw_set_c2(bbw_solver* s, const double* c2);

/* Penalty parameters tau_p, tau_u >= 0 of the fluxes (Sec. 3.1). */
bbw_status bbw_set_params(bbw_solver* s, double tau_p, double tau_u);

/*
 * Set the state q [4][K][N_p] and, if res != NULL, the RK residual register
 * res [4][K][N_p] (else res = 0), and the time t. The stage counter resets to 0.
 */
bbw_status bbw_set_state(bbw_solver* s, const double* q, const double* res, double t);

/*
 * As bbw_set_state, from caller-owned device memory in the solver's layout
 * [4][K][N_p]; dtype is BBW_F32 or BBW_F64 (converted if it differs from the
 * solver precision). res may be NULL. Ordered on the solver's stream.
 */
bbw_status bbw_set_state_device(bbw_solver* s, const void* q, const void* res, int dtype, double t);

/* Read back q (and res if non-NULL) as FP64 [4][K][N_p] and the time t (if non-NULL). */
bbw_status bbw_get_state(bbw_solver* s, double* q, double* res, double* t);

/* Copy q (and res if non-NULL) to caller-owned device memory of type dtype. */
bbw_status bbw_get_state_device(bbw_solver* s, void* q, void* res, int dtype);

/*
 * Sources. A source adds a(t) f(x) to the right-hand side of the pressure
 * equation (Eq. 1), inside the weight-adjusted bracket of Eq. (4), where the
 * spatial part f is given by degree-N Bernstein coefficients on some elements
 * and the time signature a(t) by host-given samples, one per RK stage:
 * sample 5 n + s is used at stage s of the n-th RK step counted from the last
 * bbw_set_state (its stage time is t + c_s dt, c_s from bbw_lsrk_coeffs);
 * samples past the end of amp are 0. The samples are copied; the kernels
 * read them from device memory, so any time function (a wavelet, a
 * manufactured forcing) can be driven. Setting a source replaces the
 * previous sources; nsamples = 0 removes them. Waits for the solver's stream.
 * Errors: BBW_ERR_ARG (element out of range, an element listed twice,
 * non-finite coefficients or samples, NULL with a positive count).
 */

/* One element: coeffs [N_p] on element elem, amplitude samples amp [nsamples]. */
bbw_status bbw_set_source(bbw_solver* s, int64_t elem, const double* coeffs, const double* amp,
                          int64_t nsamples);

/*
 * A forcing spread over nelem distinct elems [nelem] (caller's numbering) with
 * coefficients coeffs [nelem][N_p] and one common amplitude series
 * amp [nsamples]: f(x, t) = a(t) g(x) with g given per element.
 */
bbw_status bbw_set_forcing(bbw_solver* s, int64_t nelem, const int64_t* elems, const double* coeffs,
                           const double* amp, int64_t nsamples);

/*
 * Point source delta(x - xs) a(t) in the pressure equation: placed in the
 * lowest-numbered element whose closure contains xs, with coefficients
 * M^{-1} B(xs) / |D^k|. *elem receives that element (may be NULL).
 * Errors: BBW_ERR_ARG if xs lies outside the mesh.
 */
bbw_status bbw_set_point_source(bbw_solver* s, const double* xs, const double* amp, int64_t nsamples,
                                int64_t* elem);

/* Remove the source. */
bbw_status bbw_clear_source(bbw_solver* s);

/*
 * One LSRK stage s (0..4) with step dt: evaluates the right-hand side at
 * t + c_s dt, res = a_s res + dt rhs, q = q + b_s res. After s == 4 the
 * solver time advances by dt. Asynchronous.
 */
bbw_status bbw_stage(bbw_solver* s, int stage, double dt);

/* nsteps full RK steps (5 stages each) of size dt. Asynchronous. */
bbw_status bbw_step(bbw_solver* s, double dt, int64_t nsteps);

/*
 * CFL time step dt = cfl / (sqrt(max c^2 coefficient) * (N+1)(N+3)/3 *
 * max_{k,f} |f|/|D^k|). (The paper states no rule; this is the library's.)
 */
bbw_status bbw_cfl_dt(const bbw_solver* s, double cfl, double* dt);

/* Advance by T: nsteps = ceil(T / bbw_cfl_dt), dt = T / nsteps. Outputs may be NULL. */
bbw_status bbw_advance(bbw_solver* s, double T, double cfl, double* dt_used, int64_t* nsteps);

/* Wait for the solver's stream; returns the first pending asynchronous error. */
bbw_status bbw_sync(bbw_solver* s);

/* Current time and number of stages run since the last set_state. */
bbw_status bbw_get_time(const bbw_solver* s, double* t, int64_t* stages);

/*
 * Constants. c [N+1]: the c_j of Theorem 5.3 for P^{N+M}_N, from the
 * eigenvalues of the Bernstein mass matrix (Lemma 5.2, Corollary 1).
 * a, b, c [5]: the LSRK coefficients and stage times (any may be NULL).
 */
bbw_status bbw_projection_coeffs(int N, int M, double* c);
bbw_status bbw_lsrk_coeffs(double* a, double* b, double* c);

/*
 * Host-only self-check of the operator tables the kernels use for (N, M,
 * precision): every stencil word (one-degree reductions and elevations of
 * Eq. (12) in 3D and on faces), product gather index (Eq. 11), face map and
 * lift gather slot is recomputed by brute force over the multi-index lattice
 * and range-checked. BBW_OK, or BBW_ERR_ARG naming the first mismatch.
 * Touches no GPU.
 */
bbw_status bbw_validate_tables(int N, int M, int precision);

/*
 * The weight-adjusted update alone (the paper's timed "update kernel" minus
 * the RK part): out = P^{N+M}_N (c2_M * rhs) per element, by the product of
 * Eq. (11) and the telescoped projection of Eq. (20).
 *   rhs [K][N_p], c2 [K][M_p], out [K][N_p]: device pointers of type precision.
 *   stream: cudaStream_t (NULL = default). Asynchronous; out may not alias rhs.
 */
bbw_status bbw_wadg_update(int N, int M, int precision, int64_t K, const void* rhs,
                           const void* c2, void* out, void* stream);

/*
 * bbw_wadg_update without any device allocation. The paper has no counterpart:
 * this is a convenience of this library.
 *
 * For callers that cannot call cudaMalloc -- code running while another stream
 * is being captured into a CUDA graph, frameworks that own the whole device
 * memory pool and forbid allocations outside it, latency-critical loops that
 * must not block on the allocator. bbw_wadg_update caches its operator tables
 * in device memory it allocates on first use; this variant instead writes the
 * tables of each call into one fixed 32 KiB array in the library's static
 * device memory (present on every GPU that loads the library until the process
 * exits), passing them as the parameters of a small install kernel launched on
 * `stream` ahead of the update, so no host memory is read after the call
 * returns. It calls no cudaMalloc or cudaFree and no allocating library routine.
 * While another stream of the process is being captured in the global capture
 * mode, pass a stream other than the legacy default stream (NULL), on which no
 * work may be enqueued during such a capture.
 *   Arguments, layout and result: as bbw_wadg_update.
 *   Limit: the tables must fit in 32 KiB; every supported (N, M, precision)
 *   does except N = 9 with M = 3, which returns BBW_ERR_ARG with a message.
 *   Set-up: the first call on a device (and the first call for each
 *   (N, M, precision) on it) looks up the array's device address and sets the
 *   kernel's shared-memory attribute; make that first call before any stream
 *   capture begins.
 *   Sharing: every call uses the same array and leaves its tables there (each
 *   call overwrites the whole region it uses). Calls whose work overlaps on the
 *   GPU (different streams, or different host threads without ordering) race
 *   on the array; order them on one stream.
 */
bbw_status bbw_wadg_update_noalloc(int N, int M, int precision, int64_t K, const void* rhs,
                                   const void* c2, void* out, void* stream);

/* ------------------------------------------------------------------------
 * Receivers and the adjoint gradient with respect to c^2.
 *
 * The paper has no adjoint; these calls differentiate the discrete LSRK time
 * stepping of this library exactly (discrete adjoint, up to rounding). The
 * adjoint stage uses L(tau)^T = -M_w L(-tau) M_w^{-1} (M_w the weight-adjusted
 * mass of Eq. (4)), so it runs the forward spatial kernel with negated
 * penalties between element-local mass products.
 * ------------------------------------------------------------------------ */

/*
 * Receivers: the pressure is sampled at nrec points xyz [nrec][3] after every
 * recorded step (point evaluation of the degree-N Bernstein polynomial of the
 * containing element, lowest element index on shared faces). elems (may be
 * NULL) receives the elements [nrec]. BBW_ERR_ARG if a point is outside the
 * mesh. Discards a recorded run.
 */
bbw_status bbw_set_receivers(bbw_solver* s, int64_t nrec, const double* xyz, int64_t* elems);

/*
 * Run nsteps RK steps with step dt from the current state and time (as
 * bbw_step), keep the state every checkpoint_every steps on the device, and
 * write the receiver traces after every step to traces [nsteps][nrec] (host,
 * may be NULL). The run is kept for bbw_adjoint until the next bbw_record or
 * bbw_set_receivers. Waits for the device.
 *   checkpoint_every >= 1: memory nsteps / checkpoint_every states; the
 *   adjoint recomputes each segment once (plus 5 checkpoint_every pressure
 *   fields). checkpoint_every = 0: no checkpoints; the pressure bracket of
 *   every stage is kept instead (5 nsteps pressure fields of K N_p values in
 *   the solver's precision), so the adjoint recomputes nothing; BBW_ERR_ARG
 *   (with the sizes) if the device lacks the memory. Both give bitwise equal
 *   gradients.
 */
bbw_status bbw_record(bbw_solver* s, double dt, int64_t nsteps, int64_t checkpoint_every, double* traces);

/*
 * Gradient of J = sum_{n,r} trace_grad[n][r] * trace[n][r] over the recorded
 * run: grad_c2 [K][M_p] with respect to the c^2 coefficients, grad_q0
 * [4][K][N_p] with respect to the initial state (either may be NULL). With
 * trace_grad = trace - data this is the gradient of the L2 misfit
 * (1/2) sum (trace - data)^2. The c^2 and penalties used are the solver's
 * current ones, which must be those of the recorded run. Recomputes each
 * checkpoint segment once, keeping the five stage inputs of its steps:
 * device memory of ceil(nsteps / C) + 5 C states (C = checkpoint_every) plus
 * a few work arrays; device work of one more forward run plus the adjoint
 * stages.
 */
bbw_status bbw_adjoint(bbw_solver* s, const double* trace_grad, double* grad_c2, double* grad_q0);

/* ------------------------------------------------------------------------
 * Batches: many independent instances advanced together.
 *
 * The paper solves one mesh at a time and has no batched form; these calls
 * are a scheduling layer of this library over the same stage kernel. A batch
 * holds n instances (mesh, c^2, state, optional point source each) of uneven
 * size and degree N_i; all share M, the precision, the penalty parameters,
 * the time and dt. The instances of one degree form one bucket, a solver over
 * the disjoint union of their meshes (each instance starts on an element-group
 * boundary; detached padding tetrahedra stay at rest), so one persistent
 * launch per bucket and RK stage covers all of them. bbw_batch_step can
 * capture one RK step of all buckets into a CUDA graph and replay it; buckets
 * run as concurrent branches of that graph. Every instance evolves exactly as
 * it would alone in a bbw_solver with the same inputs and dt (same kernel, same
 * arithmetic, bitwise).
 * ------------------------------------------------------------------------ */

/*
 * Create a batch. Instance i: nverts[i] vertices vxyz[i] [nverts][3], K[i]
 * elements etov[i] [K][4] (conventions as bbw_create), degree N[i] in 1..9.
 * c^2 starts at 1, the state at 0, no sources, time 0. stream: cudaStream_t on
 * which all work of the batch is ordered (NULL: the batch creates its own,
 * since graphs cannot be captured on the legacy default stream).
 */
bbw_status bbw_batch_create(int n, const int64_t* nverts, const double* const* vxyz,
                            const int64_t* K, const int64_t* const* etov, const int* N, int M,
                            int precision, void* stream, bbw_batch** out);
void bbw_batch_destroy(bbw_batch* b);

/* Number of instances, of buckets (distinct degrees), and of elements over all
 * buckets including padding. Any pointer may be NULL. */
bbw_status bbw_batch_info(const bbw_batch* b, int* n, int* nbuckets, int64_t* elements);

/* Instance i: its degree, element count, N_p, bucket and first element in the
 * bucket's union mesh. Any output pointer may be NULL. */
bbw_status bbw_batch_member(const bbw_batch* b, int i, int* N, int64_t* K, int* Np, int* bucket,
                            int64_t* first);

/* c^2 of instance i, [K_i][M_p] (rules as bbw_set_c2). */
bbw_status bbw_batch_set_c2(bbw_batch* b, int i, const double* c2);

/* State of instance i, q and res [4][K_i][N_{p,i}] (res NULL: zero). */
bbw_status bbw_batch_set_state(bbw_batch* b, int i, const double* q, const double* res);

/* State of instance i after all enqueued work (waits; reports non-finite
 * values like bbw_sync). q or res may be NULL. */
bbw_status bbw_batch_get_state(bbw_batch* b, int i, double* q, double* res);

/* Penalty parameters of every instance (as bbw_set_params). */
bbw_status bbw_batch_set_params(bbw_batch* b, double tau_p, double tau_u);

/* Point source of instance i at xs with amplitude samples amp [nsamples]
 * (as bbw_set_point_source, searched within instance i; sample 5 n + s at
 * stage s of the n-th step since the last bbw_batch_set_time); elem (may be
 * NULL) receives its element in instance i. Setting it again replaces it. */
bbw_status bbw_batch_set_point_source(bbw_batch* b, int i, const double* xs, const double* amp,
                                      int64_t nsamples, int64_t* elem);

/* Remove every source of the batch. */
bbw_status bbw_batch_clear_sources(bbw_batch* b);

/* The smallest CFL time step over the instances (rule of bbw_cfl_dt). */
bbw_status bbw_batch_cfl_dt(const bbw_batch* b, double cfl, double* dt);

/* The CFL time step of instance i alone (rule of bbw_cfl_dt). */
bbw_status bbw_batch_member_cfl_dt(const bbw_batch* b, int i, double cfl, double* dt);

/*
 * Per-instance time steps and step budgets. dt [n] (NULL: every instance
 * steps with the dt passed to bbw_batch_step) gives instance i its own step
 * dt[i]; nsteps [n] (NULL: no budgets) stops instance i after nsteps[i] steps
 * counted from the last bbw_batch_set_time: from then on its state is carried
 * over unchanged (its groups cost one copy per stage) while the others go on.
 * All instances still take the batch's steps together, so amplitude sample
 * 5 n + s of a source is used at stage s of the batch's n-th step: sample
 * each instance's wavelet at its own stage times (t + (n + c_s) dt[i]). With
 * dt[i] the instance's CFL step (bbw_batch_member_cfl_dt) and
 * nsteps[i] = ceil(T / dt[i]), every instance reaches time T with the
 * steps it needs instead of those of the smallest CFL step of the batch.
 * Each instance evolves bitwise as its solo solver does with that dt.
 * Waits for the batch stream. Errors: BBW_ERR_ARG for a non-finite or
 * negative dt or a negative budget.
 */
bbw_status bbw_batch_set_instance_steps(bbw_batch* b, const double* dt, const int64_t* nsteps);

/* Time and steps taken of instance i (its own dt and budget). */
bbw_status bbw_batch_instance_time(const bbw_batch* b, int i, double* t, int64_t* steps);

/* Set the common time and reset the step counter (amplitude sample 0 comes next). */
bbw_status bbw_batch_set_time(bbw_batch* b, double t);

/*
 * nsteps RK steps of every instance with step dt, asynchronous on the batch
 * stream. use_graph != 0: each step is one replay of a CUDA graph of the whole
 * step (built on first use per state-buffer parity and rebuilt when dt or the
 * penalty parameters change); 0: the same launches enqueued directly.
 */
bbw_status bbw_batch_step(bbw_batch* b, double dt, int64_t nsteps, int use_graph);

/*
 * Choose the batch's launch schedule by timing: every candidate (buckets as
 * concurrent graph branches or one after another; persistent grids of 1/2,
 * 1 or 2 times the solo grid) runs `steps` graph-replayed steps and the
 * fastest is kept for later bbw_batch_step calls. The trial steps use dt = 0,
 * which leaves the state and the time unchanged (res is reset, as at any
 * step's first stage). schedule (may be NULL) receives the chosen candidate
 * (0 = default: concurrent branches, solo grids) and ms_per_step (may be
 * NULL) its time per step. Waits for the batch.
 */
bbw_status bbw_batch_autotune(bbw_batch* b, int steps, int* schedule, double* ms_per_step);

/* Wait for the batch and surface non-finite values (as bbw_sync). */
bbw_status bbw_batch_sync(bbw_batch* b);

/* Time and number of steps since the last bbw_batch_set_time (or creation). */
bbw_status bbw_batch_get_time(const bbw_batch* b, double* t, int64_t* steps);

/* ---------------------------------------------------------------------------
 * Elastic solver (Sec. 2.2): the velocity-stress system
 *
 *     rho dv/dt = sum_i A_i^T d sigma/dx_i,   C^{-1} dsigma/dt = sum_i A_i dv/dx_i
 *
 * with the isotropic constitutive matrix C(lambda, mu) and the matrix-weighted
 * weight-adjusted update of Eq. (ewadg). One bbw_elastic_stage() is one LSRK
 * stage over all elements in one fused GPU kernel: the Bernstein derivatives
 * (Sec. 4), penalty fluxes
 *     F_v = 1/2 A_n^T [[sigma]] + tau_v/2 A_n^T A_n [[v]],
 *     F_s = 1/2 A_n [[v]] + tau_s/2 A_n A_n^T [[sigma]]    (A_n = sum_i n_i A_i),
 * the factored lift, the products with the degree-M media polynomials and the
 * telescoped projection of Eq. (20) (ten scalar projections per element:
 * three with rho^{-1}, one with lambda, six with mu), and the LSRK update.
 *
 *  - State arrays are [9][K][N_p], fields (v_x, v_y, v_z, s_xx, s_yy, s_zz,
 *    s_yz, s_xz, s_xy) in the multi-index order above.
 *  - Media arrays (rho^{-1}, lambda, mu) are [K][M_p] Bernstein coefficients
 *    of degree M; rho^{-1} coefficients must be > 0, lambda and mu >= 0.
 *  - Walls are traction-free mirrors: sigma+ = -sigma, v+ = v.
 *  - Ownership, streams and errors follow the acoustic solver; the mesh rules
 *    and limits of bbw_create apply.
 * ------------------------------------------------------------------------- */

/* Create an elastic solver on the mesh (as bbw_create); media default to
 * rho^{-1} = lambda = mu = 1, penalties tau_v = tau_s = 1, state 0. */
bbw_status bbw_elastic_create(int64_t nverts, const double* vxyz, int64_t K, const int64_t* etov, int N, int M,
                              int precision, void* cuda_stream, bbw_elastic** out);
/* Wait for the solver's stream and free it (NULL: no-op). */
void bbw_elastic_destroy(bbw_elastic* s);
/* Sizes and precision (any pointer may be NULL). */
bbw_status bbw_elastic_info(const bbw_elastic* s, int64_t* K, int* N, int* M, int* Np, int* Mp, int* precision);
/* Media: rho_inv, lam, mu each [K][M_p]. BBW_ERR_NONPOS_C2 if a rho^{-1}
 * coefficient is <= 0, a lambda or mu coefficient < 0, or any is not finite. */
bbw_status bbw_elastic_set_media(bbw_elastic* s, const double* rho_inv, const double* lam, const double* mu);
/* Penalty parameters (finite, >= 0); tau = 0 gives central fluxes. */
bbw_status bbw_elastic_set_params(bbw_elastic* s, double tau_v, double tau_s);
/* State q [9][K][N_p], RK residual res (NULL: zero) and time t. */
bbw_status bbw_elastic_set_state(bbw_elastic* s, const double* q, const double* res, double t);
/* Read back q and res ([9][K][N_p], either may be NULL) and t; waits and
 * reports asynchronous failures as bbw_elastic_sync. */
bbw_status bbw_elastic_get_state(bbw_elastic* s, double* q, double* res, double* t);
/* State from caller-owned device memory [9][K][N_p] of type dtype (32 | 64),
 * res may be NULL (zero); ordered on the solver's stream. */
bbw_status bbw_elastic_set_state_device(bbw_elastic* s, const void* q, const void* res, int dtype, double t);
/* Copy q (and res if non-NULL) to caller-owned device memory [9][K][N_p] of
 * type dtype, ordered on the solver's stream. */
bbw_status bbw_elastic_get_state_device(bbw_elastic* s, void* q, void* res, int dtype);
/* One LSRK stage s in 0..4 with step dt (asynchronous). */
bbw_status bbw_elastic_stage(bbw_elastic* s, int stage, double dt);
/* nsteps full RK steps of size dt (asynchronous). */
bbw_status bbw_elastic_step(bbw_elastic* s, double dt, int64_t nsteps);
/* dt = cfl / (c_p,max (N+1)(N+3)/3 max_f |f|/|D|), c_p,max^2 bounded by the
 * largest element value of max(lambda + 2 mu) max(rho^{-1}) (coefficients). */
bbw_status bbw_elastic_cfl_dt(const bbw_elastic* s, double cfl, double* dt);
/* Advance by T with nsteps = ceil(T / dt_cfl) steps of dt = T / nsteps
 * (dt_used, nsteps may be NULL). */
bbw_status bbw_elastic_advance(bbw_elastic* s, double T, double cfl, double* dt_used, int64_t* nsteps);
/* Wait for the solver's stream; BBW_ERR_NONFINITE if a stage produced a NaN
 * or Inf since the last check. */
bbw_status bbw_elastic_sync(bbw_elastic* s);
/* Time and number of stages since the last bbw_elastic_set_state. */
bbw_status bbw_elastic_get_time(const bbw_elastic* s, double* t, int64_t* stages);

#ifdef __cplusplus
}
#endif

#endif /* BBWADG_H */
