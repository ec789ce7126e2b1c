/*
 * pyrdg.h - C ABI of libpyrdg.so: time-explicit discontinuous Galerkin for the
 * first-order acoustic wave system on meshes of vertex-mapped pyramids, after
 * Chan & Warburton, "Orthogonal bases for vertex-mapped pyramids".
 *
 * What one call computes (Sec. 4.3, rho = kappa = 1, so c = 1 and
 * tau_p = tau_u = tau): for every element K, with the semi-nodal basis of
 * Lemma 3 and the cubature of Sec. 4.1,
 *     M dp/dt   = -( sum_m S^m u_m + L^f F_p ),
 *     M du_m/dt = -( S^m p          + L^f F_{u_m} ),
 *     F_p = 1/2 (n.[[u]] - tau [[p]]),   F_u = 1/2 n ([[p]] - tau n.[[u]]),
 * [[q]] = q+ - q-. M is diagonal in the semi-nodal basis (Lemma 3):
 *     M_{ijk,ijk} = J(a_i^k, b_j^k) w_i^k w_j^k C_k,  C_k = 2/(2k+3),
 * and is applied as that diagonal; no per-element matrix is stored or inverted.
 * Time stepping is the 5-stage 2N-storage RK4 of Carpenter and Kennedy that
 * Sec. 4.1 cites (Alg. 3 of Sec. 4.2 is its stage update).
 *
 * Conventions shared by every call:
 *  - Reference pyramid (Sec. 2): r, s in [-1, -t], t in [-1, 1]; collapsed
 *    coordinates a, b, c in [-1, 1] with r = (1+a)(1-c)/2 - 1,
 *    s = (1+b)(1-c)/2 - 1, t = c.
 *  - Element vertices (EToV row, 0-based into `vertices`): v1..v4 the base
 *    quadrilateral with (v2-v1) x (v4-v1) pointing toward the apex v5, v3
 *    opposite v1 (the images of (-1,-1,-1), (1,-1,-1), (1,1,-1), (-1,1,-1),
 *    (-1,-1,1)).
 *  - State layout: row-major [K][nf][Np]; nf = 4 fields (p, u, v, w) for the wave
 *    equation, nf = 1 (u) for advection (pyr_dg_num_fields); Np =
 *    (N+1)(N+2)(2N+3)/6 coefficients of the semi-nodal basis per field, in
 *    the order n = k(k+1)(2k+1)/6 + j(k+1) + i for phi_ijk =
 *    l_i^k(a) l_j^k(b) ((1-c)/2)^k P_{N-k}^{(2k+3,0)}(c), l^k the Lagrange
 *    polynomials at the (k+1) Gauss-Legendre points. Element type is double
 *    for PYR_DG_F64 handles and float for PYR_DG_F32 handles.
 *  - Errors: every int-returning call returns PYR_DG_OK (0) or a negative
 *    code; pyr_dg_last_error() then gives a message (thread-local). No C++
 *    exception crosses this boundary. There is no CPU fallback: without a
 *    usable CUDA device, calls that compute return PYR_DG_ERR_CUDA.
 *  - Streams: work is enqueued on opts.stream (a cudaStream_t; NULL means the
 *    legacy default stream). Calls that return host data synchronise that
 *    stream; the others return once the work is enqueued.
 */
#ifndef PYRDG_H
#define PYRDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PYR_DG_OK = 0,
  PYR_DG_ERR_BAD_ARG = -1,        /* null pointer, size out of range, unknown enum */
  PYR_DG_ERR_BAD_MESH = -2,       /* J <= 0, vertex index out of range, non-conforming face */
  PYR_DG_ERR_UNSUPPORTED_N = -3,  /* N outside [PYR_DG_MIN_N, PYR_DG_MAX_N] */
  PYR_DG_ERR_CUDA = -4,           /* CUDA runtime error (message has the CUDA string) */
  PYR_DG_ERR_NO_MEMORY = -5,      /* host or device allocation failed */
  PYR_DG_ERR_TIMEOUT = -6         /* a bounded wait inside a kernel gave up (results invalid) */
};

enum { PYR_DG_MIN_N = 1, PYR_DG_MAX_N = 7 };
enum { PYR_DG_F64 = 0, PYR_DG_F32 = 1 };
enum { PYR_DG_BC_WALL = 0, PYR_DG_BC_FREE = 1 };
enum { PYR_DG_HOST = 0, PYR_DG_DEVICE = 1 };
enum { PYR_DG_WAVE = 0, PYR_DG_ADVECTION = 1 };
enum { PYR_DG_MODAL = 0, PYR_DG_NODAL = 1 };

typedef struct pyr_dg pyr_dg; /* opaque handle, owned by the library */

typedef struct pyr_dg_opts {
  int precision;  /* PYR_DG_F64 (state and arithmetic in double) or PYR_DG_F32
                     (state and stage arithmetic in float; geometry and the
                     error norm still in double) */
  int bc;         /* PYR_DG_BC_WALL: rigid wall n.u = 0 (mirror p+ = p-,
                     u+ = u- - 2(n.u-)n); PYR_DG_BC_FREE: free surface p = 0
                     of Sec. 4.3 (p+ = -p-, u+ = u-) */
  double tau;     /* flux penalty of Sec. 4.3: 1 = upwind, 0 = central; >= 0 */
  void* stream;   /* cudaStream_t for all work of this handle; NULL = default */
  int device;     /* CUDA device ordinal; -1 = the calling thread's current device */
  int equation;   /* PYR_DG_WAVE: the acoustic system (p, u, v, w), 4 fields.
                     PYR_DG_ADVECTION: u_t + div(beta u) = 0 of Sec. 4.1, 1 field, with
                     the alpha-flux ((beta_n - alpha|beta_n|)/2)(u+ - u-), alpha = tau
                     (1 upwind, 0 central); needs periodic = 1 */
  double beta[3]; /* advection velocity (PYR_DG_ADVECTION) */
  int periodic;   /* 1: the box [box_lo, box_hi]^3 is periodic: faces on opposite boundary
                     planes are neighbours (their vertices must coincide modulo the period) */
  double box_lo, box_hi;
  int basis;      /* PYR_DG_MODAL: the state holds semi-nodal coefficients (layout above).
                     PYR_DG_NODAL: the nodal variant of Sec. 4.4.1 (wave equation, F64
                     only): the state holds each field's values at Np nodes, the
                     Lagrange basis at them spans the same space, so the discrete
                     solution is the same function. Nodes (pyr_dg_host_nodal_points):
                     layer m = 0..N at c = the m-th of the N+1 Gauss-Lobatto-Legendre
                     (GLL) points, carrying the (N+1-m) x (N+1-m) GLL grid in (a, b)
                     (the apex layer one node at (0, 0, 1)); ordered by layer, then b,
                     then a. M^{-1} is applied as V M_phi^{-1} V^T, V the Vandermonde of
                     the semi-nodal basis at the nodes; triangle faces are integrated
                     with the nodal face mass matrix, the (possibly non-planar) base with
                     its Gauss-Legendre rule. */
} pyr_dg_opts;

/* Fill *opts with: F64, wall, tau = 1, stream NULL, device -1, wave equation,
 * beta = (1, 0, 0), not periodic, box [0, 1], modal basis. */
void pyr_dg_default_opts(pyr_dg_opts* opts);

/* The nodal set of the nodal variant at degree N (host only, no GPU needed):
 * abc receives Np x 3 doubles, the collapsed coordinates (a, b, c) of each node
 * in state order (see pyr_dg_opts.basis). */
int pyr_dg_host_nodal_points(int N, double* abc);

/* Build a solver for one mesh (Sec. 2 vertex maps, Sec. 4.1 cubature).
 * vertices: host, Nv x 3 doubles, row-major (copied).
 * EToV:     host, K x 5 int32 indices into vertices (copied), order as above.
 * N:        polynomial degree, PYR_DG_MIN_N..PYR_DG_MAX_N.
 * opts:     may be NULL for the defaults.
 * On success *out owns device memory for the state, the LSRK residual, face
 * traces, per-element geometric factors, the mass diagonal and the face
 * connectivity; the state is zero and the time is 0. Faces are matched by
 * their vertex sets; every shared face must carry coincident cubature
 * points (conforming mesh), else PYR_DG_ERR_BAD_MESH. Unshared faces take
 * the boundary condition. Synchronises the stream. */
int pyr_dg_setup(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                 const pyr_dg_opts* opts, pyr_dg** out);

/* Sizes of a handle: elements K, degree N, coefficients per field Np,
 * face cubature points per element Nfc = 5(N+1)^2, precision. Any pointer may be NULL. */
int pyr_dg_info(const pyr_dg* h, int64_t* K, int* N, int* Np, int* Nfc, int* precision);

/* Fields per element of the state: 4 (wave) or 1 (advection). */
int pyr_dg_num_fields(const pyr_dg* h, int* nf);

/* L2 projection (volume rule of Sec. 4.1, diagonal mass of Lemma 3) of the
 * exact standing wave at time t0 into the state; sets the time to t0 and
 * zeroes the LSRK residual. 'wall': p = cos(pi x)cos(pi y)cos(pi z)cos(sqrt3 pi t),
 * u = sin(pi x)cos(pi y)cos(pi z)sin(sqrt3 pi t)/sqrt3 (cyclic), for [0,1]^3;
 * 'free': the resonant cavity of Sec. 4.3 on [-1,1]^3. Advection: u0(x - beta t) with
 * u0 = sin(2 pi X) cos(2 pi Y) sin(2 pi Z), X = (x - box_lo)/(box_hi - box_lo). Asynchronous. */
int pyr_dg_project(pyr_dg* h, double t0);

/* Copy a state in (set) or out (get). q: K*4*Np elements of the handle's
 * type, layout above; `where` = PYR_DG_HOST or PYR_DG_DEVICE says where q
 * lives. set_state also sets the time to t and zeroes the LSRK residual.
 * Both synchronise the stream. */
int pyr_dg_set_state(pyr_dg* h, const void* q, int where, double t);
int pyr_dg_get_state(pyr_dg* h, void* q, int where);

/* Stage the input of the next step from host memory without waiting: q_host (K*4*Np
 * elements of the handle's type, layout above) is copied on a copy stream of the handle
 * into a second device buffer, so the copy overlaps work already enqueued (the current
 * step). The next pyr_dg_step waits on the device for that copy, makes it the state, sets
 * the time to t and zeroes the LSRK residual, then steps. Until then every other call
 * (pyr_dg_error, pyr_dg_get_state, pyr_dg_rhs, ...) sees the current state;
 * pyr_dg_set_state and pyr_dg_project drop a staged state, and a later stage replaces an
 * earlier one. The paper has no counterpart (it is host-device plumbing for callers that
 * feed a new state every step). Ownership: the caller keeps q_host. From page-locked memory
 * the copy is asynchronous: q_host must not change until pyr_dg_sync returns, or a call
 * that synchronises the stream (pyr_dg_error, pyr_dg_get_state) returns after the step that
 * consumed it. Pageable memory also works, without the overlap. The first call allocates
 * the second buffer (same size as the state); PYR_DG_ERR_NO_MEMORY if that fails. */
int pyr_dg_stage_state(pyr_dg* h, const void* q_host, double t);

/* Right-hand side dU/dt = -M^{-1}(volume + surface terms) of the state q
 * (device pointer, K*4*Np of the handle's type) into rhs (device pointer,
 * same size, must not alias q). Uses the handle's trace buffer as scratch;
 * does not touch the handle's own state. Asynchronous. */
int pyr_dg_rhs(pyr_dg* h, const void* q_dev, void* rhs_dev);

/* Allocation-free variant of pyr_dg_rhs. The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory when
 * they call it, for example code whose device memory is all owned by another
 * allocator (a framework's caching pool, a fixed arena) or a phase in which
 * allocating would stall or is forbidden by the caller's own rules.
 * Same inputs, outputs and result as pyr_dg_rhs (q_dev -> rhs_dev, device
 * pointers of K*4*Np elements of the handle's type, no aliasing), but the face
 * traces go to a static device array of PYR_DG_NOALLOC_SCRATCH_BYTES bytes
 * compiled into the library instead of the handle's trace buffer. The call
 * performs no cudaMalloc, cudaFree or other allocating routine.
 *  - Size limit: K * Nfc * 4 * sizeof(element) must not exceed
 *    PYR_DG_NOALLOC_SCRATCH_BYTES (8 MiB: e.g. 2097 pyramids at N = 4 in
 *    double); larger handles get PYR_DG_ERR_BAD_ARG and a message.
 *  - The array exists on every GPU that loads the library, until the process
 *    exits. pyr_dg_setup looks up the array's device address
 *    (cudaGetSymbolAddress) with the handle's device current and caches it
 *    per device; under lazy module loading that lookup is also when the
 *    driver places the array on the device, so it happens in setup, where
 *    allocating is allowed, and never inside this call for a handle whose
 *    setup succeeded. (Only if that lookup failed in setup does this call
 *    retry it; such a first call should come before any stream capture.)
 *  - Every call shares the one array per device and it keeps the last call's
 *    contents. Each call writes every entry it reads before reading it, so
 *    nothing needs clearing, but calls whose work overlaps on the GPU (other
 *    streams, other handles, other threads) race on it: serialise them.
 * Asynchronous, on the handle's stream. */
enum { PYR_DG_NOALLOC_SCRATCH_BYTES = 8 << 20 };
int pyr_dg_rhs_noalloc(pyr_dg* h, const void* q_dev, void* rhs_dev);

/* Advance the handle's state nsteps LSRK4 steps of size dt (> 0); each step
 * is 5 stages, each stage one trace launch and one fused
 * volume + flux + lift + M^{-1} + update launch. Advances the time by
 * nsteps*dt. Asynchronous. */
int pyr_dg_step(pyr_dg* h, int nsteps, double dt);

/* L2 error of the state against the exact standing wave at the current time,
 * integrated in double with (N+3)-point rules (Gauss-Legendre in a, b,
 * Gauss-Jacobi (2,0) in c), over all four fields; l2_rel divides by the L2
 * norm of the exact solution. Either pointer may be NULL. Synchronises. */
int pyr_dg_error(pyr_dg* h, double* l2_abs, double* l2_rel);
/* The exact fields are S(x) times a time factor: S = products of cos/sin(pi sc x),
 * sc = 1 (wall) or 1/2 (free surface), times cos or sin of sqrt3 pi sc t. Let P be the
 * projection onto each element's polynomial space under the error rule's inner product;
 * that rule integrates the mass matrix exactly, so M is the diagonal of Lemma 3. Then,
 * per field, the squared error is sum_i M_ii (u_i - T s_i)^2 + T^2 |P S - S|^2 with s the
 * coefficients of P S, and only the time factor T changes between calls. On a wave
 * handle the second pyr_dg_error stores s, M in double and the mesh sums of |P S - S|^2
 * and |S|^2: 5 K Np doubles of device memory (plus 4 per error block), allocated only
 * when that is at most a quarter of the free device memory, and freed by
 * pyr_dg_destroy. That call and later ones then read only the coefficients. Without
 * the store (the first call, or when it does not fit) the call evaluates U_h and the
 * exact fields at the error-rule points. Both give the same value up to rounding. */

/* L2 distance between two states of this handle (device pointers, K x nf x Np
 * elements of the handle's type, any may alias): d2 = sum over elements, fields
 * and modes of M_ii (qa_i - qb_i)^2 and n2 = the same of M_ii qb_i^2, summed in
 * double. The semi-nodal basis is orthogonal on every element (Lemma 3) and the
 * volume rule integrates the mass matrix exactly, so these are the squared L2
 * norms of the difference and of qb over the mesh, M_ii = 1 / (the stored
 * M^{-1} entry). Either output pointer may be NULL. Synchronises. */
int pyr_dg_l2_diff(pyr_dg* h, const void* qa_dev, const void* qb_dev, double* d2, double* n2);

/* enable = 0: free the stored factors and evaluate the exact fields at every call;
 * enable != 0 (the default): store them at the second pyr_dg_error from now when
 * they fit.
 * Synchronises the handle's stream when it frees the store. */
int pyr_dg_set_error_cache(pyr_dg* h, int enable);

/* Time step dt = cfl / (C_N max_K |dK|/|K|), C_N = 2(N+1)(N+3)/3, the
 * spectral-radius fit of Sec. 4.3. Synchronises. */
int pyr_dg_dt_cfl(pyr_dg* h, double cfl, double* dt);

/* Current simulation time of the handle. */
int pyr_dg_time(const pyr_dg* h, double* t);

/* Single-precision stage with the level mixing (the c direction of the volume
 * term, Sec. 4.2 Alg. 1 recast as small matrices per level) on the tensor cores:
 * per element and RK stage, each (a, b) point's mixing inputs form one row of an
 * M = 128 operand and one chain of tcgen05.mma kind::tf32 (FP32 accumulation in
 * tensor memory) applies all mixing matrices at once, with the 3-term split
 * A_hi B_hi + A_hi B_lo + A_lo B_hi for about FP32 accuracy. enable != 0 selects
 * it, 0 the CUDA-core kernel (the default). FP32 wave handles only, else
 * PYR_DG_ERR_BAD_ARG. One element per CTA; measured slower than the CUDA-core
 * kernel on GB300 (the mixing is 2 to 8 terms wide, and each element waits for
 * its MMAs). Its completion waits are bounded: pyr_dg_sync returns
 * PYR_DG_ERR_TIMEOUT if one gave up since the last check. */
int pyr_dg_set_tensor_mixing(pyr_dg* h, int enable);

/* Face traces on the tensor cores (Alg. 3's interpolation of the state to the face points,
 * batched over elements), for the stepping of modal wave handles (pyr_dg_step). The trace map
 * Phi_f (mode n at face point g, Nfc x Np) is the same for every element and field, so the
 * traces of a tile of elements are one product with the state's rows (element x field, the
 * state's own layout) and K = Np modes. Phi_f is taken in FP64 from the trace kernel applied
 * to unit states and prepared on the host when the traces are first enabled.
 *  - FP32 handles: T = U Phi_f^T over 32 elements (M = 128 rows), tcgen05.mma kind::tf32 with
 *    the 3-term split A_hi B_hi + A_hi B_lo + A_lo B_hi (about FP32 accuracy), FP32
 *    accumulation in tensor memory. Every stage runs the stage kernel without its trace passes,
 *    then this kernel writes the new state's traces into the other half of the trace pair.
 *    Handles of at least 40,000 elements start with it at N = 2..7, where it measured faster;
 *    smaller meshes and N = 1 start without it. The operator takes about 2 Nfc Np floats.
 *  - FP64 handles at N = 2..4 (Nfc <= 128 face points, Np <= 102 modes): Phi_f U^T over 8
 *    elements with FP64 accuracy: Phi_f's rows and the state's rows are cut into 8 exact
 *    balanced base-128 digits against each row's largest exponent (BF16 operands of
 *    tcgen05.mma kind::f16), the 36 digit products of each level s = i + j <= 7 are summed
 *    exactly as integers below 2^22 in FP32 accumulators, and integer arithmetic with one
 *    integer-to-FP64 conversion recombines the 8 levels into FP64. Each trace is within
 *    15.1 K 2^-58 + 2^-55 of 2^(E+F-2044) (E, F:
 *    the two rows' largest biased exponents, K = Np terms) plus half an ulp of the exact dot
 *    product, below FP64's own worst-case rounding bound for such a sum. It replaces the FP64
 *    trace kernel before each fused stage; pyr_dg_rhs and the projection keep that kernel.
 *    Handles of at least 40,000 elements start with it at N = 3, 4, where it measured
 *    faster (a tie at N = 2). The operator takes 16 * 128 * Np(padded to 16) + 512 bytes.
 * enable != 0 selects these traces, 0 the CUDA-core paths. Other handles (advection, the nodal
 * basis, FP64 at N = 1 or N >= 5) return PYR_DG_ERR_BAD_ARG. Completion waits are bounded as
 * for pyr_dg_set_tensor_mixing. */
int pyr_dg_set_tensor_traces(pyr_dg* h, int enable);

/* Whether the handle's stepping currently computes the face traces on the tensor cores
 * (pyr_dg_set_tensor_traces or the handle's default): *enabled = 1 or 0. */
int pyr_dg_get_tensor_traces(const pyr_dg* h, int* enabled);

/* Wait for all work enqueued by this handle, staged state copies included. */
int pyr_dg_sync(pyr_dg* h);

/* Per-kernel timing of pyr_dg_step: with enable != 0, every stage kernel that
 * pyr_dg_step launches is bracketed by CUDA events on the handle's stream
 * (a few microseconds of overhead per launch); enable = 0 turns it off. Either
 * call discards what was recorded before. */
int pyr_dg_profile(pyr_dg* h, int enable);

/* Totals since the last pyr_dg_profile call: device milliseconds and launch
 * counts of the trace kernel and of the fused volume/flux/lift/M^{-1}/update
 * kernel. FP32 handles run one stage kernel that also writes the new state's
 * traces; their trace kernel runs only when the traces are not current (after
 * setup, set_state, project or rhs). Synchronises the stream. Any pointer may be NULL. */
int pyr_dg_profile_read(pyr_dg* h, double* trace_ms, int64_t* trace_launches, double* rhs_ms,
                        int64_t* rhs_launches);

/* Free the handle and its device memory (synchronises first). NULL is a no-op. */
void pyr_dg_destroy(pyr_dg* h);

/* Message for the last failing call on this thread ("" if none). */
const char* pyr_dg_last_error(void);

/* ---- batched form: many independent meshes of uneven sizes and degrees ----
 * The meshes of one degree are held as one disjoint-union mesh, so every RK
 * stage is one persistent launch per distinct degree over all of its meshes,
 * with each element using its own mesh's time step; one pyr_dg_batch_step
 * call is a captured CUDA graph (captured on first use for a given nsteps,
 * replayed afterwards). For PYR_DG_F32 batches the persistent grid of each
 * degree is autotuned at setup (timed on the all-zero initial state). The
 * state, time and errors are per mesh. opts applies to every mesh; with
 * opts->stream NULL the batch creates its own non-blocking stream (graph
 * capture needs one), reported by pyr_dg_batch_stream. */
typedef struct pyr_dg_batch pyr_dg_batch;

/* vertices[i] (Nv[i] x 3 doubles), EToV[i] (K[i] x 5 int32) and N[i] describe
 * mesh i, i < nmesh; all host arrays, copied. Errors as pyr_dg_setup. */
int pyr_dg_batch_setup(int nmesh, const double* const* vertices, const int64_t* Nv, const int32_t* const* EToV,
                       const int64_t* K, const int* N, const pyr_dg_opts* opts, pyr_dg_batch** out);
/* Number of meshes, of degree groups (= launches per stage), total elements and
 * total degrees of freedom (sum of K * 4 * Np). Any pointer may be NULL. */
int pyr_dg_batch_info(const pyr_dg_batch* b, int* nmesh, int* ngroups, int64_t* total_K, int64_t* total_dofs);
/* Degree, element count, launch grid and elements per CTA of degree group
 * `group` < ngroups. For FP32 the grid (persistent CTAs) and the elements per CTA
 * (1, 2, 4 or 8) are autotuned at setup on that group; FP64 launches one CTA per
 * element. Any out pointer may be NULL. */
int pyr_dg_batch_group_info(const pyr_dg_batch* b, int group, int* N, int64_t* K, int* stage_blocks,
                            int* elems_per_block);
/* Project the exact standing wave at t0 into every mesh; sets every mesh's time to t0. */
int pyr_dg_batch_project(pyr_dg_batch* b, double t0);
/* Per-mesh CFL time steps (as pyr_dg_dt_cfl) into dt[nmesh]. */
int pyr_dg_batch_dt_cfl(const pyr_dg_batch* b, double cfl, double* dt);
/* How the batch runs an RK stage (chosen at setup by timing both on the zero state):
 * single_launch = 1: one persistent kernel per stage runs every degree group (FP32
 * batches of 2..8 groups; the group's share of its CTAs is tuned from each group's
 * measured cost), launches_per_stage = 1; single_launch = 0: one persistent launch per
 * degree group, the groups on parallel branches of the step's CUDA graph,
 * launches_per_stage = the group count. Either pointer may be NULL. */
int pyr_dg_batch_launch_mode(const pyr_dg_batch* b, int* single_launch, int* launches_per_stage);
/* Override that choice: single_launch != 0 selects the single kernel per stage
 * (PYR_DG_ERR_BAD_ARG where it is not available), 0 the per-group launches. */
int pyr_dg_batch_set_launch_mode(pyr_dg_batch* b, int single_launch);

/* Advance every mesh nsteps LSRK4 steps of its own dt[i] > 0. Asynchronous. */
int pyr_dg_batch_step(pyr_dg_batch* b, int nsteps, const double* dt);
/* Per-mesh L2 errors (as pyr_dg_error) into l2_abs[nmesh], l2_rel[nmesh]
 * (either may be NULL). Synchronises. */
int pyr_dg_batch_error(pyr_dg_batch* b, double* l2_abs, double* l2_rel);
/* Copy the state of mesh `mesh` (K[mesh] x 4 x Np elements) to q on the host or
 * device (`where`). Synchronises. */
int pyr_dg_batch_get_state(pyr_dg_batch* b, int mesh, void* q, int where);
int pyr_dg_batch_sync(pyr_dg_batch* b);
void* pyr_dg_batch_stream(const pyr_dg_batch* b);
void pyr_dg_batch_destroy(pyr_dg_batch* b);

/* ---- host-side builder queries (no GPU needed; used to test the builder) ---- */

/* n-point Gauss-Jacobi rule for weight (1-x)^alpha (1+x)^beta on [-1,1]
 * (Newton iteration on P_n^{(alpha,beta)}), nodes ascending into x[n],
 * weights into w[n]. 1 <= n <= 64, alpha, beta > -1. */
int pyr_dg_host_gauss_jacobi(int n, double alpha, double beta, double* x, double* w);

/* Face connectivity the setup would build, without a GPU. mapP: host,
 * K*5*(N+1)^2 int64; entry (e*Nfc + g) is the global face-point index
 * (e'*Nfc + g') matched to point g of element e, or e*Nfc + g itself on a
 * boundary face. Face-point order per element: face 0 base (a_p, b_q),
 * g = p + (N+1) q; faces 1..4 = {b=-1, a=+1, b=+1, a=-1} at (x_e, c_m),
 * g = f(N+1)^2 + e + (N+1) m with x_e the Gauss-Legendre coordinate along the
 * base edge and c_m the Gauss-Jacobi (1,0) coordinate toward the apex.
 * nboundary (may be NULL) receives the number of boundary faces. */
int pyr_dg_host_connectivity(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                             int64_t* mapP, int64_t* nboundary);

/* As pyr_dg_host_connectivity, with the box [box_lo, box_hi]^3 periodic: faces on
 * opposite boundary planes are matched as neighbours (cubature points compared
 * modulo the period). */
int pyr_dg_host_connectivity_periodic(const double* vertices, int64_t Nv, const int32_t* EToV, int64_t K, int N,
                                      double box_lo, double box_hi, int64_t* mapP, int64_t* nboundary);

/* Measured FMA throughput of this GPU in TFLOP/s (2 flops per FMA) for
 * precision PYR_DG_F64 or PYR_DG_F32: a register-only kernel of independent
 * FMA chains over every SM, timed with CUDA events. Synchronises the
 * default stream; used as the ALU roofline peak. */
int pyr_dg_fma_peak(int precision, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* PYRDG_H */
