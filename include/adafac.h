/*
 * adafac.h -- C ABI of the GB300 adAFAC multigrid library.
 *
 * The library solves the vertex-based d-linear finite element discretisation
 * of  -div(eps grad u) = f  (Eq. 1 of Murray & Weinzierl, "Stabilised
 * Asynchronous Fast Adaptive Composite Multigrid using Additive Damping",
 * arXiv:1903.10367) on the unit square/cube with zero Dirichlet data, on a
 * regular spacetree of depth L with 3:1 refinement per dimension (Sec. 2.1).
 * Levels are numbered l = 1 (coarsest level with unknowns, l_min) .. L
 * (finest, l_max); level l has n_l = 3^l cells per dimension and
 * (n_l + 1)^d vertices, of which (n_l - 1)^d interior ones are unknowns.
 *
 * One call of adafac_cycle() runs additive multigrid cycles in which every
 * level at once computes its residual, one damped Jacobi step and (adAFAC-Jac)
 * the auxiliary damping equation on the next coarser level; all corrections
 * are prolonged and summed (Algorithm 1, Eq. 9).  Everything after the input
 * copy runs in the library's CUDA kernels on the caller's stream.
 *
 * Array layout (all vertex arrays): C order, x fastest, then y, then z; an
 * array of a level with n cells holds (n+1)^d entries including the boundary
 * ring.  Per-cell arrays hold n^d entries in the same order.
 *
 * Conventions of every entry point:
 *   - returns an adafac_status; never aborts, never throws;
 *   - a failing call leaves a message retrievable with adafac_last_error();
 *   - calls on one handle are not thread-safe; different handles are
 *     independent;
 *   - device work is enqueued on the handle's stream; functions documented
 *     as "synchronises" wait for that stream.
 */
#ifndef ADAFAC_H
#define ADAFAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adafac_handle_s* adafac_handle;

typedef enum {
  ADAFAC_OK = 0,
  ADAFAC_ERR_INVALID_ARG = 1,   /* bad pointer, size, option or state       */
  ADAFAC_ERR_OOM = 2,           /* workspace too small / allocation failed  */
  ADAFAC_ERR_DIVERGED = 3,      /* residual non-finite or grew > 1e6 x r_0  */
  ADAFAC_ERR_TIMEOUT = 4,       /* reserved for bounded device waits        */
  ADAFAC_ERR_CUDA = 5,          /* a CUDA runtime call failed               */
  ADAFAC_ERR_NOT_CONVERGED = 6  /* adafac_solve hit max_cycles              */
} adafac_status;

/* Regular spacetree: dim in {2, 3}, 1 <= depth (L), ((3^L+1)^dim must fit in
 * 2^31 vertices).  The coarsest level taking part in the cycles is
 * adafac_options.lmin (1 by default, the paper's benchmark setting,
 * Sec. 2.1). */
typedef struct {
  int dim;
  int depth;
} adafac_tree;

enum {
  ADAFAC_VARIANT_ADDITIVE = 0,  /* plain additive multigrid, Eq. 2          */
  ADAFAC_VARIANT_JAC = 1,       /* adAFAC-Jac, Algorithm 1 / Eq. 9          */
  ADAFAC_VARIANT_PI = 2,        /* adAFAC-PI, Algorithm 2                   */
  ADAFAC_VARIANT_EXP = 3        /* Eq. 2 with omega_add(l) = omega_exp^(L-l) */
};
enum { ADAFAC_TRANSFER_DLINEAR = 0, ADAFAC_TRANSFER_BOXMG = 1 };
enum { ADAFAC_PRECISION_FP64 = 0, ADAFAC_PRECISION_MIXED = 1 };
enum { ADAFAC_RTILDE_TRUNCATED = 0, ADAFAC_RTILDE_EXACT = 1 };
enum { ADAFAC_FORM_CS = 0, ADAFAC_FORM_FAS = 1 };

typedef struct {
  int variant;        /* ADAFAC_VARIANT_*, default JAC                        */
  int transfer;       /* ADAFAC_TRANSFER_*: d-linear or BoxMG (Sec. 2.4)      */
  int precision;      /* FP64: every step in FP64.  MIXED: the cycles run in
                         FP32 on the correction equation A e = r, grouped into
                         refinement steps whose residual r = b - A u and update
                         u += e are FP64 (iterative refinement).              */
  int rtilde;         /* smoothed restriction R~ (Sec. 3.2, option 1):
                         TRUNCATED = omega (M^-1 A_{eps=1} P)^T cut to the 5^d
                         support of P; EXACT = omega R A_l M_l^-1             */
  int form;           /* CS: coarse residuals r_l = R r_{l+1};  FAS: injected
                         coarse solutions and FAS/HTMG right-hand sides
                         (Eq. 4).  FAS requires precision FP64.               */
  int inner_cycles;   /* MIXED: FP32 cycles per FP64 refinement step (>= 1)  */
  double omega;       /* Jacobi damping, default 0.6 (Sec. 5)                */
  double omega_tilde; /* damping-equation Jacobi damping, default 0.6        */
  double omega_exp;   /* base of exponential damping (VARIANT_EXP)           */
  int path;           /* ADAFAC_PATH_AUTO: fused kernels where the configuration
                         allows them (3-D, scalar eps, d-linear, MIXED, CS form,
                         JAC/ADDITIVE/EXP with truncated R~), else one kernel
                         per level and step; ADAFAC_PATH_LEVELWISE: always the
                         latter (same arithmetic, other summation order).
                         In MIXED precision the per-level kernels are shaped
                         like the grids (a thread per vertex or coarse vertex,
                         compile-time stencil offsets and weights);
                         ADAFAC_PATH_GENERIC selects the generic per-level
                         kernels instead (a linear index decoded per vertex,
                         a warp per coarse vertex in the restriction): the
                         same steps, another summation order.  FP64 cycles
                         always use the generic kernels.
                         ADAFAC_PATH_BATCHED (MIXED precision, CS form, any
                         variant but JAC with exact R~): a whole refinement
                         step -- the FP64 residual and its norm, inner_cycles
                         FP32 cycles of Alg. 1 and u += e -- is one launch in
                         which a cluster of CTAs runs the steps of the cycle
                         one after another, separated by cluster barriers.
                         The request server runs the steps of all its running
                         BATCHED requests of one dimension and cluster size
                         in one launch, a cluster per request; every vertex
                         is computed the same way whatever the batch or the
                         cluster size, so a request's iterates do not depend
                         on the requests it runs with.  AUTO takes this path
                         too for MIXED solves it covers whose finest grid has
                         at most 1024 vertices (2-D depth <= 3, 3-D depth <=
                         2) and that the fused 3-D kernels do not take.       */
  int coarse_op;      /* ADAFAC_COARSE_GALERKIN (default): A_{l-1} =
                         P_l^T A_l P_l (Sec. 2.2); ADAFAC_COARSE_REDISCRETISED:
                         the d-linear FEM operator of level l-1 with the eps of
                         a coarse cell the mean of its 3^dim children          */
  int lmin;           /* coarsest level taking part in the cycles, 1 (default)
                         .. depth; levels below lmin are not used (Sec. 5 adds
                         correction levels one by one below the finest)      */
} adafac_options;

enum { ADAFAC_PATH_AUTO = 0, ADAFAC_PATH_LEVELWISE = 1, ADAFAC_PATH_GENERIC = 2,
       ADAFAC_PATH_BATCHED = 3 };
enum { ADAFAC_COARSE_GALERKIN = 0, ADAFAC_COARSE_REDISCRETISED = 1 };

/* Fills *opt with the defaults: JAC, d-linear, FP64, truncated R~, CS,
 * inner_cycles 24, omega = omega_tilde = 0.6, omega_exp = 0.5, path AUTO,
 * Galerkin coarse operators, lmin 1. */
adafac_status adafac_default_options(adafac_options* opt);

/* Device bytes a handle for (tree, opt) needs.  Pass at least this much
 * 256-byte aligned device memory to adafac_setup, or NULL there to let the
 * library allocate it. */
adafac_status adafac_workspace_size(const adafac_tree* tree,
                                    const adafac_options* opt, size_t* bytes);

/* Builds the hierarchy (Sec. 2.1-2.4): load vector b_L = h^d f (lumped mass),
 * fine operator from per-cell eps, for l = L..2 the prolongation P_l
 * (d-linear or BoxMG) and the Galerkin operator A_{l-1} = P_l^T A_l P_l, the
 * inverse diagonals, and the smoothed-restriction stencil.  All in FP64; MIXED
 * keeps FP32 copies for the cycles.  The iterate starts at u = 0.
 *
 *   eps   per finest-level cell (3^L)^dim doubles, or one double if
 *         eps_is_scalar; every value must be > 0
 *   f     right-hand side at every finest-level vertex, (3^L+1)^dim doubles
 *         (boundary entries ignored), or NULL for f = 0
 *   inputs_on_device  0: eps and f are host pointers (copied, may be pageable);
 *                     1: device pointers (copied device-to-device)
 *   workspace / workspace_bytes  caller-owned device memory of at least
 *         adafac_workspace_size() bytes that outlives the handle, or NULL
 *         (library allocates and frees it)
 *   stream  cudaStream_t for all device work of this handle (NULL: default)
 *
 * Inputs are copied; the caller may free them once the call returns.
 * Synchronises.  On failure *out is NULL and nothing stays allocated. */
adafac_status adafac_setup(const adafac_tree* tree, const double* eps,
                           int eps_is_scalar, const double* f,
                           int inputs_on_device, const adafac_options* opt,
                           void* workspace, size_t workspace_bytes,
                           void* stream, adafac_handle* out);

/* Enqueues n_cycles >= 0 cycles (Algorithm 1 / Eq. 9 or the chosen variant).
 * FP64: each cycle updates u.  MIXED: the cycles act on the FP32 correction
 * equation in groups of at most inner_cycles; each group starts from the FP64
 * residual of u and ends with u += e, so u is current when the call returns.
 * Asynchronous. */
adafac_status adafac_cycle(adafac_handle h, int n_cycles);

/* Runs cycles until ||r||_h / ||r_0||_h <= rel_tol (Eq. 10, r_0 = b for the
 * initial u = 0 of setup, or the residual at the last adafac_set_solution /
 * adafac_reset) or max_cycles cycles.  The test runs on the device; batches of
 * cycles after convergence return immediately.  *cycles_done receives the
 * number of cycles applied, *rel the final normalised residual (either may be
 * NULL).  Returns ADAFAC_ERR_NOT_CONVERGED or ADAFAC_ERR_DIVERGED when the
 * tolerance was not met.  Synchronises. */
adafac_status adafac_solve(adafac_handle h, double rel_tol, int max_cycles,
                           int* cycles_done, double* rel);

/* Residual of the current iterate in FP64: *abs = ||b - A u||_h (Eq. 10)
 * and *rel = *abs / ||r_0||_h.  Either pointer may be NULL.  Synchronises. */
adafac_status adafac_residual_norm(adafac_handle h, double* rel, double* abs);

/* Copies the current fine-level iterate u ((3^L+1)^dim doubles including the
 * boundary values) to dst (host if dst_on_device == 0, else device).
 * Synchronises. */
adafac_status adafac_solution(adafac_handle h, double* dst, int dst_on_device);

/* Sets the iterate u from src (same layout; boundary entries are ignored and
 * keep the Dirichlet values) and makes its residual the new r_0.
 * Synchronises. */
adafac_status adafac_set_solution(adafac_handle h, const double* src,
                                  int src_on_device);

/* Sets the Dirichlet values: the boundary entries of g ((3^L+1)^dim doubles,
 * host if g_on_device == 0, else device; interior entries ignored) become
 * the boundary of u and stay fixed; the interior of u is kept and its
 * residual becomes the new r_0.  The setups of Sec. 5 prescribe u = 1 on
 * x_2 = 0 and 0 elsewhere (setup starts with zero values).  Requires the
 * correction-scheme form (INVALID_ARG for FAS).  Synchronises. */
adafac_status adafac_set_boundary(adafac_handle h, const double* g, int g_on_device);

/* Resets u = 0 inside (the Dirichlet values on the boundary), r_0 := the next
 * residual evaluated, and the history.
 * Asynchronous (a device kernel resets the control block). */
adafac_status adafac_reset(adafac_handle h);

/* Poll limit of the bounded device-side waits on h.  The fused 3-D sweeps
 * stage their planes by asynchronous copies and wait for each on a shared
 * memory barrier; a wait gives up after `polls` polls or 2 s of device time,
 * whichever comes first (default 4194304 polls).  A wait that gives up stores
 * nothing of its step, its block leaves, the kernels after it in the batch
 * return at entry, and the next synchronising call returns
 * ADAFAC_ERR_TIMEOUT naming where the first wait gave up (adafac_last_error).
 * polls = 0 makes every wait give up before its first poll, so the timeout
 * path can be exercised without a copy that never lands; the iterate then
 * keeps its value from before the batch.  adafac_reset clears the fault.
 * The paper has no counterpart (its code runs on CPUs).  Handles off the
 * fused path have no such waits and ignore the value.  INVALID_ARG for
 * polls < 0.  Synchronises (cycles already enqueued keep the old limit). */
adafac_status adafac_set_wait_limit(adafac_handle h, long long polls);

/* CTAs per instance of the batched path (ADAFAC_PATH_BATCHED).  Performance
 * extension with no counterpart in the paper: the cluster of CTAs that runs
 * a handle's refinement steps.  Setup picks one CTA when the FP32 vectors fit
 * into 100 KB of shared memory (they are then held there), else a power of
 * two from the size of the finest grid (about 8 vertices per thread, at most
 * 16, or 8 where the device cannot place clusters of 16); every choice
 * computes the same iterates bit for bit.  adafac_set_batch_cluster takes a
 * power of two in 1 .. that limit (INVALID_ARG otherwise, or when the handle
 * does not run the batched path); adafac_batch_cluster writes the current
 * value to *ctas.
 * Neither call touches the device. */
adafac_status adafac_set_batch_cluster(adafac_handle h, int ctas);
adafac_status adafac_batch_cluster(adafac_handle h, int* ctas);

/* Inspection of internal per-level arrays (for tests and diagnostics).
 * field: ADAFAC_FIELD_*; level: 1..L.  Copies the array as doubles to dst
 * (host or device) and writes its length to *count (pass dst = NULL to query
 * the length only).  Vectors have (n_l+1)^d entries; P has 2^d entries per
 * vertex of level l (entry c weights the corner with offset bit j = (c>>j)&1
 * along dimension j, x = 0, of the owning coarse cell
 * floor(min(i/3, n_{l-1}-1))), stored entry-major (c * V + vertex);
 * STENCIL has 3^d entries per vertex, entry s = sum_j (o_j+1) 3^j, stored
 * entry-major.  Vectors of the most recent cycle: R residual r_l, BT damping
 * right-hand side b~_l, G combined correction g_l = c_l - c~_l, T prolonged
 * sum t_l.  Synchronises. */
enum {
  ADAFAC_FIELD_U = 0,       /* fine iterate (level L only)                 */
  ADAFAC_FIELD_B = 1,       /* fine load vector (level L only)             */
  ADAFAC_FIELD_R = 2,
  ADAFAC_FIELD_BT = 3,
  ADAFAC_FIELD_G = 4,
  ADAFAC_FIELD_T = 5,
  ADAFAC_FIELD_P = 6,       /* prolongation l-1 -> l (l >= 2, BoxMG only)  */
  ADAFAC_FIELD_STENCIL = 7, /* Galerkin stencil of level l < L             */
  ADAFAC_FIELD_INVDIAG = 8  /* 1 / diag(A_l)                               */
};
adafac_status adafac_get_field(adafac_handle h, int field, int level,
                               double* dst, int dst_on_device, size_t* count);

/* Normalised residual history: entry k is ||r_k||_h / ||r_0||_h of the k-th
 * residual evaluated on the device since setup/reset (one per FP64 cycle,
 * one per refinement step in MIXED).  Copies up to max_entries doubles to the
 * host array dst and the number available to *count.  Synchronises. */
adafac_status adafac_history(adafac_handle h, double* dst, int max_entries,
                             int* count);

/* Number of kernel launches the library has enqueued on this handle since
 * setup (setup kernels excluded). */
adafac_status adafac_launch_count(adafac_handle h, uint64_t* count);

/* Per-kernel device timing with CUDA events recorded on the handle's stream
 * around every launch of the kernels below (for roofline measurements; the
 * events add a few microseconds per launch).  adafac_timing(h, 1) starts
 * recording and clears the accumulators, adafac_timing(h, 0) stops.
 * adafac_timing_read synchronises and returns, for one kernel kind, the summed
 * device time in milliseconds and the number of timed launches since the
 * last adafac_timing(h, 1). */
enum {
  ADAFAC_KERNEL_FINE_RESIDUAL = 0, /* residual of the finest level (cycle)   */
  ADAFAC_KERNEL_FINE_UPDATE = 1,   /* fine-level update x += c_L + P q      */
  ADAFAC_KERNEL_FINE_RESTRICT = 2, /* restriction from the finest level (on
                                      the 3-D uniform path: the first up-pass
                                      of a refinement step)                 */
  ADAFAC_KERNEL_REFINE = 3,        /* FP64 refinement residual (MIXED)      */
  ADAFAC_KERNEL_FINE_DOWN = 4,     /* 3-D uniform path: down-pass, the fine
                                      update with its residual recomputed  */
  ADAFAC_KERNEL_FINE_UP = 5,       /* 3-D uniform path: up-pass, residual +
                                      restriction + damping right-hand side */
  ADAFAC_KERNEL_FINE_DOWN_U = 6,   /* 3-D uniform path: last down-pass of a
                                      refinement step, which also adds the
                                      correction to the FP64 iterate       */
  ADAFAC_KERNEL_BATCH_STEP = 7,    /* path BATCHED: a whole refinement step */
  ADAFAC_KERNEL_KINDS = 8
};
adafac_status adafac_timing(adafac_handle h, int enable);
adafac_status adafac_timing_read(adafac_handle h, int kind, double* total_ms,
                                 int* launches);

/* ---- Autotuner of tile and launch shapes ---------------------------------
 *
 * Performance extension; the paper has no counterpart (its cycle runs on a
 * CPU spacetree traversal).  adafac_autotune times candidate shapes of the
 * handle's dominant fine-level kernels on the handle's own arrays and keeps
 * the fastest (a candidate replaces the default only when it is at least 2 %
 * faster):
 *   path 1, the fused 3-D sweeps (MIXED, scalar eps, d-linear, 3-D): the
 *     number of balanced slabs along z into which the up-passes split the
 *     interior coarse planes and the down-passes the interior fine planes
 *     (sweep_nz, sweep_nz_down: every count whose slabs are 3 to 24 coarse
 *     planes thick);
 *   path 2, the grid-shaped level kernels (MIXED otherwise, path not
 *     GENERIC): the block shape of the fine residual and of the fine update
 *     (res_bx x res_by, upd_bx x upd_by threads from 32x8, 64x4, 32x4,
 *     128x2, 64x2, 256x1) and the length of the residual's z columns
 *     (res_zr planes, 0 = the size rule; 3-D only);
 *   path 0: nothing to tune (FP64 precision or path GENERIC).
 * Every shape computes the same values: solutions, norms and cycle counts do
 * not change.  Each candidate is timed over `repeats` launches (1..1000)
 * after one untimed launch.  Results are kept per process, device and
 * problem shape (dim, depth, path, eps kind, transfer, variant, lmin): a later
 * handle of the same shape takes them without timing (cached = 1).
 * The call synchronises the handle's stream, runs only on the handle's
 * arrays (no device memory is allocated), and resets the cycle state (control block,
 * history, correction buffers; not the iterate u): call it after setup and
 * before cycling.  *out is a caller-owned record, filled on success.
 * Returns INVALID_ARG (null argument, repeats out of range) or CUDA. */
typedef struct {
  int path;            /* 0 nothing tuned, 1 fused 3-D sweeps, 2 level kernels */
  int cached;          /* 1: taken from an earlier tuning of the same shape   */
  int sweep_nz;        /* path 1: slabs along z of the up-passes              */
  int sweep_nz_down;   /* path 1: slabs along z of the down-passes            */
  int res_bx, res_by;  /* path 2: threads per block of the fine residual      */
  int res_zr;          /* path 2: planes per thread column (0 = size rule)    */
  int upd_bx, upd_by;  /* path 2: threads per block of the fine update        */
  int candidates;      /* launch shapes timed                                 */
  double us_default;   /* one launch each of the tuned kernels, default shapes, us */
  double us_tuned;     /* the same with the chosen shapes, us                 */
} adafac_tuning;
adafac_status adafac_autotune(adafac_handle h, int repeats, adafac_tuning* out);

/* sqrt(h^dim * sum over the interior vertices i of r_i^2), r = b - A u, where
 * A is the uniform d-linear finite-element stencil of -div(eps grad u) with
 * scalar eps and h = 3^-depth, on a regular grid of 3^depth cells per axis in
 * `dim` = 2 or 3 dimensions, computed WITHOUT ALLOCATING device memory.
 * The paper has no counterpart.  This entry exists for callers that cannot
 * allocate: a process whose device memory is fully committed to resident
 * workspaces, or code that must not pay the device-wide synchronisation of a
 * device free.
 *   u     device array of (3^depth + 1)^dim doubles, x fastest, boundary ring
 *         included.  The stencil of a vertex next to the boundary reads the
 *         ring, so the ring must hold the Dirichlet values (zero for
 *         homogeneous problems); caller-owned, read only.
 *   b     device array of the same shape; only its interior values are read
 *         (its ring is ignored); caller-owned, read only.
 *   norm  device pointer to one double, written asynchronously on `stream`
 *         (a cudaStream_t, NULL = legacy default stream).
 * The per-block partial sums live in a fixed device array of the library
 * (4096 doubles, one per 16384 vertices), so (3^depth + 1)^dim must be at most
 * 4096 * 16384 = 67,108,864 vertices; larger trees return INVALID_ARG without
 * launching.  Nothing in that array needs to start at zero: every partial the
 * norm reads is written by the same call.
 * The array exists once per CUDA context.  The first call in each context
 * (also after a cudaDeviceReset, which makes a new context) looks up its
 * address with cudaGetSymbolAddress; make that first call outside any stream
 * capture (under capture it returns CUDA).  All calls in a context share the
 * array: calls that overlap in time (other streams, other host threads) race
 * on it and may return wrong norms; order them on one stream.
 * Returns INVALID_ARG (bad dim/depth/eps, null pointer, tree too large) or
 * CUDA (launch failure, or the first call of a context made under capture);
 * adafac_last_error is not updated by this call. */
adafac_status adafac_residual_norm_static(int dim, int depth, double eps, const double* u,
                                         const double* b, double* norm, void* stream);

/* ---- Request server: continuous batching of independent solves ---------
 *
 * Serving extension; the paper has no counterpart.  A server owns one device
 * pool of device_bytes, n_streams CUDA streams on the device current at
 * creation and host threads of its own.  Submitted requests wait in a queue until
 * their workspace (adafac_workspace_size) fits into the free part of the pool
 * and one of max_running slots is free; the request in slot i runs on stream
 * i mod n_streams (n_streams >= max_running gives each its own stream);
 * requests with workspaces up to 64 MiB use high-priority streams.  An
 * admitted request is set up, then runs batches of cycles (inner_cycles for
 * MIXED, 8 for FP64) until ||r||_h / ||r_0||_h <= rel_tol (Eq. 10) or
 * max_cycles; requests on different streams overlap on the device, and
 * requests submitted while others run are admitted as memory and slots free
 * up.  At completion the solution is copied to host memory and the
 * request's device memory returns to the pool.  Every function may be called
 * from any host thread. */
typedef struct adafac_server_s* adafac_server;

enum {
  ADAFAC_REQUEST_PENDING = 0,  /* queued, not yet admitted   */
  ADAFAC_REQUEST_RUNNING = 1,  /* admitted: in setup, cycles or completion */
  ADAFAC_REQUEST_DONE = 2,     /* converged; solution ready  */
  ADAFAC_REQUEST_FAILED = 3    /* ended with status != OK    */
};

typedef struct {
  int state;          /* ADAFAC_REQUEST_*                                      */
  int status;         /* final status code: OK when DONE, else the reason;
                         NOT_CONVERGED still delivers the last iterate        */
  int cycles;         /* cycles applied                                        */
  double rel;         /* last evaluated ||r||_h / ||r_0||_h                    */
  double queue_ms;    /* submission -> admission (-1 while queued)             */
  double latency_ms;  /* submission -> solution in host memory (-1 until then) */
} adafac_request_info;

/* Allocates the pool (one cudaMalloc) and starts the worker.  OOM if the
 * pool cannot be allocated; INVALID_ARG for n_streams outside 1..256 or
 * max_running < 1.  Requests run on up to 2 n_streams streams plus one per
 * batched launch group: start the process with CUDA_DEVICE_MAX_CONNECTIONS
 * set to 32 (read when the CUDA context is created; the driver's default is
 * 8), so that streams do not share hardware work queues and a small
 * request's kernels do not wait behind a large one's (measured on the
 * serving mix at 0.8 x saturated load: p50 latency 86 ms with 8 queues, 31
 * ms with 32). */
adafac_status adafac_server_create(size_t device_bytes, int n_streams, int max_running,
                                   adafac_server* out);

/* Queues a solve; arguments as adafac_setup (host inputs, copied before the
 * call returns) plus the tolerance and the cycle limit (>= 1).  *ticket
 * identifies the request.  OOM when the request's workspace exceeds the
 * whole pool (it could never run). */
adafac_status adafac_submit(adafac_server s, const adafac_tree* tree, const double* eps,
                            int eps_is_scalar, const double* f, const adafac_options* opt,
                            double rel_tol, int max_cycles, int64_t* ticket);

/* State, cycles, residual and timings of a request (non-blocking). */
adafac_status adafac_poll(adafac_server s, int64_t ticket, adafac_request_info* info);

/* For a request that has ended: copies its solution ((3^L+1)^dim doubles)
 * into host memory dst (unless dst is NULL or the request produced none),
 * forgets the ticket and returns the request's final status.  INVALID_ARG
 * for unknown tickets and for requests still queued or running. */
adafac_status adafac_fetch(adafac_server s, int64_t ticket, double* dst);

/* Requests queued / admitted and not yet ended, and pool bytes in use. */
adafac_status adafac_server_stats(adafac_server s, int* pending, int* running,
                                  size_t* bytes_in_use);

/* Stops the worker (running requests end FAILED), frees the pool and
 * forgets every ticket.  Synchronises. */
adafac_status adafac_server_destroy(adafac_server s);

/* ---- Adaptive spacetrees (static trees; moving refinement by transfer) ---
 *
 * Sec. 2.1 and 2.3: level 1 exists in full (l_min = 1); a level-l cell that
 * exists is cut into 3^dim children where refine[l-1][cell] != 0 (l = 1 ..
 * depth-1; 3^(l*dim) bytes per level, x fastest; flags of cells that do not
 * exist are ignored).  The leaf cells carry the d-linear element of
 * -div(eps grad u); eps of a leaf cell coarser than the finest level is the
 * mean of the finest cells it covers.  The unknowns are the values at the
 * leaf nodes (the corners of the leaf cells); hanging nodes carry none, their
 * values follow d-linearly from the coarser level.  Level l's shape
 * functions are the pagodas of its active vertices (interior vertices whose
 * 2^dim level-l cells all exist), a generating system over the adaptive grid:
 * level l sees r_l = Phi_l^T (b - K u) with K the leaf stiffness, A_l =
 * Phi_l^T K Phi_l, M_l = diag(A_l), and a cycle is Eq. 9 on that system
 * (the options' variant, rtilde, omega, omega_tilde, omega_exp and lmin as
 * for regular trees; the truncated R~ acts on level l's residual held on its
 * full grid, zero at inactive positions).  The load is lumped per leaf cell:
 * each corner of a leaf cell of width h takes h^dim / 2^dim f.  Dirichlet
 * values are zero.
 *   eps  host, one value (eps_is_scalar) or 3^(depth*dim) values (finest
 *        cells, x fastest)
 *   f    host, (3^depth + 1)^dim values at the finest-level positions, or
 *        NULL (zero)
 * Inputs are copied during the call.  The handle owns its device memory
 * (allocated here), runs on `stream` (cudaStream_t; NULL = legacy default).
 * Two engines compute the same cycles.  By default every level works on its
 * full grid (the tiles of it that meet an existing cell): r_l is the chain
 * rho_l = W_l + P^T rho_{l+1} of the levels' leaf-cell residuals W_l, the
 * corrections return by T_l = g_l + P T_{l-1}, and M_l comes from the
 * Galerkin element matrices collapsed level by level.  Path GENERIC, and the
 * exact R~ of Jac, use Phi_l and K as sparse matrices instead.  Precision
 * FP64 runs every step in FP64; MIXED (grid engine only) runs refinement
 * steps: the FP64 leaf-cell residuals of every level and their norm, then
 * inner_cycles FP32 cycles on the correction equation, then u += e in FP64.
 * Returns INVALID_ARG for a bad tree or options (BoxMG transfers,
 * rediscretised coarse operators and MIXED on the sparse-matrix engine are
 * not available), OOM when an allocation fails. */
typedef struct adafac_adaptive_s* adafac_adaptive;
adafac_status adafac_adaptive_setup(int dim, int depth, const uint8_t* const* refine,
                                    const double* eps, int eps_is_scalar, const double* f,
                                    const adafac_options* opt, void* stream,
                                    adafac_adaptive* out);

/* Enqueues n_cycles >= 0 cycles (Eq. 9 on the generating system; MIXED:
 * refinement steps of at most inner_cycles cycles).  Asynchronous. */
adafac_status adafac_adaptive_cycle(adafac_adaptive h, int n_cycles);

/* Eq. 10 over the vertices of the nodal space (every position that is an
 * active vertex of some level, tested with that level's pagoda, h of that
 * level): *abs = ||b - K u||_h, *rel = *abs / ||r_0||_h (r_0: the residual
 * at setup or at the last adafac_adaptive_set_solution).  Either may be NULL.
 * Synchronises. */
adafac_status adafac_adaptive_residual_norm(adafac_adaptive h, double* rel, double* abs);

/* Cycles until the normalised residual is <= rel_tol or max_cycles cycles ran;
 * NOT_CONVERGED / DIVERGED as adafac_solve.  The grid engine tests the norm
 * on the device before every cycle (MIXED: before every refinement step)
 * and synchronises after every 8 cycles (MIXED: every step); the sparse-matrix
 * engine synchronises every cycle. */
adafac_status adafac_adaptive_solve(adafac_adaptive h, double rel_tol, int max_cycles,
                                    int* cycles_done, double* rel);

/* The leaf nodes: *count receives their number; idx (or NULL) their
 * finest-level grid indices x + (3^depth + 1) (y + (3^depth + 1) z),
 * ascending -- the order of the values of the solution calls. */
adafac_status adafac_adaptive_nodes(adafac_adaptive h, int64_t* idx, int64_t* count);

/* The iterate at the leaf nodes (host dst, count values).  Synchronises. */
adafac_status adafac_adaptive_solution(adafac_adaptive h, double* dst);

/* Sets the iterate from host src (count values, zero at boundary nodes for
 * the zero Dirichlet data) and makes its residual the new r_0.  Synchronises. */
adafac_status adafac_adaptive_set_solution(adafac_adaptive h, const double* src);

/* Moving refinement (Sec. 5): sets dst's iterate from src, a handle on
 * another tree of the same dim and depth.  The vertices of dst's tree take
 * the value of src's function at their position (d-linear interpolation in
 * the src leaf cell that holds them, so new vertices are interpolated), and
 * the function of dst's space with those vertex values is rebuilt level by
 * level from the coarsest (vertices hanging in dst's tree take the
 * interpolation of their coarse cell).  dst's r_0 becomes src's, so the
 * normalised residual keeps its reference across moves.  INVALID_ARG for
 * trees of another shape; synchronises both streams. */
adafac_status adafac_adaptive_transfer(adafac_adaptive dst, adafac_adaptive src);

/* Level vectors of the active vertices of a level (ascending grid index of
 * the level's (3^level + 1)^dim grid): FIELD_ACTIVE their grid indices,
 * FIELD_R r_l of the last residual evaluation (a cycle or a norm), FIELD_BT
 * b~_l and FIELD_G the combined correction g_l of the last cycle,
 * FIELD_INVDIAG 1 / M_l.  *count receives the number of active vertices;
 * dst (host, or NULL) the values.  Synchronises. */
enum { ADAFAC_FIELD_ACTIVE = 9 };
adafac_status adafac_adaptive_level(adafac_adaptive h, int field, int level, double* dst,
                                    int64_t* count);

/* Message of the last failing call on an adaptive handle (empty for NULL). */
const char* adafac_adaptive_last_error(adafac_adaptive h);

/* Releases the handle and its device memory.  Synchronises. */
adafac_status adafac_adaptive_destroy(adafac_adaptive h);

/* Message of the last failing call on h (or of the last failing setup when
 * h is NULL).  The pointer stays valid until the next call on h. */
const char* adafac_last_error(adafac_handle h);

/* Releases the handle and the workspace it allocated.  Synchronises. */
adafac_status adafac_destroy(adafac_handle h);

#ifdef __cplusplus
}
#endif

#endif /* ADAFAC_H */
