/*
 * igamg — multigrid-preconditioned CG for multi-patch isogeometric Poisson problems on
 * one GB300 (sm_103a).  C ABI.
 *
 * Method (Hofer & Takacs, "A parallel multigrid solver for multi-patch Isogeometric
 * Analysis"): the Poisson model problem of Sec. 2 (-Laplace u = f, u = 0 on Gamma_D,
 * du/dn = 0 on Gamma_N) discretised by a fully matching multi-patch spline space V_l
 * (Eq. vh), grid levels l = 0..L by uniform refinement (Sec. 3), the cycle of
 * Algorithm 1 with the additive Schwarz smoother of Eq. additive, an exact coarsest solve,
 * used as the preconditioner of PCG (Sec. 4, Sec. 5).
 *
 * Conventions shared by every entry point
 *  - All calls return an igamg_status and never abort or throw.  After an error the
 *    context stays valid for igamg_free() and igamg_last_error().
 *  - Device vectors are FP64, length N_l (igamg_num_dofs), in the library's global dof
 *    numbering of level l (igamg_dof_map).  They are caller-owned device memory; every
 *    call runs on the stream given to igamg_setup and returns without synchronising it
 *    unless stated.  Level index l: 0 = coarsest, L = num_levels-1 = finest; -1 = finest.
 *  - Host arrays passed to igamg_setup are read during the call only.
 *  - The context owns the grid hierarchy (band coefficients, smoother bases, transfer
 *    tables, coarse factor) and its device workspaces; only igamg_free releases them.
 *  - A context is used by one host thread at a time (its work buffers and captured CUDA
 *    graphs are per context); different contexts may be used concurrently from different
 *    threads, as the batch and server layers below do.
 *  - igamg_solve synchronises the stream once per PCG iteration (the convergence test
 *    reads the residual norm on the host) and at its end.
 */
#ifndef IGAMG_H
#define IGAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IGAMG_OK = 0,
  IGAMG_ERR_ARG = 1,          /* NULL pointer, bad size, bad level, bad enum          */
  IGAMG_ERR_GEOMETRY = 2,     /* non-matching patches, tagged interface, bad vertices */
  IGAMG_ERR_UNSUPPORTED = 3,  /* non-uniform knots, geometry degree != 1, ...         */
  IGAMG_ERR_OOM = 4,          /* device allocation failed                              */
  IGAMG_ERR_CUDA = 5,         /* a CUDA runtime call failed                           */
  IGAMG_ERR_NUMERIC = 6,      /* NaN/Inf in PCG scalars, Cholesky/eigen breakdown      */
  IGAMG_ERR_NOT_CONVERGED = 7,/* max_iter reached; x and res->relres are filled        */
  IGAMG_ERR_TIMEOUT = 8
} igamg_status;

/* Side tags (Sec. 2: Gamma_D / Gamma_N).  Side s of a patch is parameter direction s/2 at
 * end s%2, order -x,+x,-y,+y,-z,+z.  AUTO: interface when another patch has the same side
 * (same corner vertices), otherwise Dirichlet.  An interface side must be tagged AUTO. */
enum { IGAMG_SIDE_AUTO = 0, IGAMG_SIDE_DIRICHLET = 1, IGAMG_SIDE_NEUMANN = 2 };

enum { IGAMG_FP64 = 0, IGAMG_FP32 = 1, IGAMG_BF16 = 2 };

/* Multi-patch problem (Sec. 2, Eq. matching).  Patch k has, per direction j, a spline
 * degree degree[k*dim+j] and an open uniform knot vector at the finest level (num_knots
 * entries, concatenated over k and j in that order in `knots`).  The geometry map G_k is
 * multilinear: geo_degree = 1 and geo_num_ctrl = 2 in every direction, and geo_ctrl holds,
 * per patch, its 2^dim corner points (dim coordinates each), corner c = sum_j c_j 2^j with
 * c_j the end of direction j.  Patches must be fully matching (common sides have the same
 * corners and the same knot vectors).  Level 0 has m_L / 2^L intervals per direction. */
typedef struct {
  int dim;                 /* 2 or 3                                          */
  int num_patches;         /* K >= 1                                          */
  const int* degree;       /* [K*dim]   p >= 1                                 */
  const int* num_knots;    /* [K*dim]                                          */
  const double* knots;     /* sum(num_knots) values                            */
  const int* geo_degree;   /* [K*dim]   must be 1                              */
  const int* geo_num_ctrl; /* [K*dim]   must be 2                              */
  const double* geo_ctrl;  /* [K * 2^dim * dim]                                */
  const int* side_bc;      /* [K*2*dim] IGAMG_SIDE_*                           */
  int num_levels;          /* L+1 >= 1                                         */
} igamg_problem;

/* Solver parameters; defaults are the paper's (Sec. 5): tau = 0.25, sigma = h^{-2}/0.2,
 * one pre- and one post-smoothing step, V-cycle. */
typedef struct {
  double tau;          /* smoother damping (Eq. sm)                                 */
  double sigma_scale;  /* sigma = sigma_scale * h_l^{-2} in the interior smoother      */
  int nu;              /* smoothing steps before and after the coarse correction       */
  int mu;              /* 1 = V-cycle, 2 = W-cycle (Algorithm 1)                      */
  int max_iter;        /* PCG iteration limit (inner iterations in total for mixed)   */
  int precision;       /* IGAMG_FP64: PCG in FP64.  IGAMG_FP32 / IGAMG_BF16: FP64
                          iterative refinement around a PCG whose vectors, smoother
                          contractions and transfers are FP32 and whose band
                          coefficients are FP32 / BF16 (FP32 accumulation); the
                          eigendecompositions, the refinement residual and the coarse
                          solve stay FP64                                            */
  double inner_tol;    /* mixed precision: relative reduction of each inner PCG (1e-4) */
  int fd_engine;       /* patch-interior FD contractions: 0 = automatic (the autotuner's
                          choice per level, else tensor cores on 2D interiors of >= 96
                          dofs per direction), 1 = FMA pipes in the working precision,
                          2 = tensor cores on every level (FP64: exact BF16 digit slices
                          with integer recombination; BF16 variant: BF16 operands),
                          3 = one block per 2D interior of <= 32 x 32 (all four
                          contractions in shared memory), FMA GEMMs elsewhere,
                          4 = 2D interiors in two launches over blocks of 8 rows (each
                          fusing two of the products), FMA GEMMs in 3D               */
  int graphs;          /* 1: each PCG iteration after the first is captured once as a
                          CUDA graph and replayed (same launches, same order, same
                          results); 0: launched one by one                            */
  int apply_engine;    /* stiffness apply above the coarsest level (2D): 0 = a Kronecker
                          sum of the 1D stiffness and mass when every patch is a
                          rectangle (no band storage), stored bands otherwise;
                          1 = stored bands always                                     */
  int autotune;        /* with fd_engine 0: time the FD candidates of every level once at
                          setup (FMA tile factors 1, 2, 4; tensor cores on interiors of
                          >= 32; the one-block kernel on 2D interiors of <= 32; the
                          row-block kernel on 2D interiors) and keep
                          the fastest; choices are cached per interior shape for the life
                          of the process                                               */
  int batch_engine;    /* igamg_setup_batch: 0 = lockstep when every problem is in its scope
                          (2D, rectangle patches, FP64, V-cycle): one launch per cycle step
                          over all problems, one graph replay per PCG iteration of the whole
                          batch; otherwise, and with 1, worker streams (whole single solves
                          on concurrent streams)                                        */
} igamg_options;

/* Result of a solve.  The first five fields are the problem statement's result record;
 * outer_iters, added for the precision variant, comes last so that their layout is kept. */
typedef struct {
  int iters;           /* PCG iterations performed (inner iterations for mixed)       */
  double relres;       /* ||b - A x||_2 / ||b - A x_0||_2 at exit                      */
  double t_setup_ms;   /* igamg_setup wall time (host + device, synchronised)          */
  double t_assemble_ms;/* part of setup spent assembling the level matrices           */
  double t_solve_ms;   /* this solve, device-synchronised wall time                    */
  int outer_iters;     /* FP64 refinement steps (1 for FP64)                          */
} igamg_result;

typedef struct igamg_ctx igamg_ctx;

/* Fills *opt with the defaults above (max_iter = 500, precision FP64). */
igamg_status igamg_default_options(igamg_options* opt);

/* Sec. 5 setup phase (dof mappers, refinement and transfers, piece-local smoothers,
 * coarse solver) plus the assembly of every level's patch matrices (Eq. model:bil) on
 * the device.  `opt` may be NULL (defaults).  `cuda_stream` is a cudaStream_t or NULL
 * for the legacy default stream; the context issues all its work there.  Uses the
 * current CUDA device.  On success *out owns a new context; on failure *out is NULL. */
igamg_status igamg_setup(const igamg_problem* problem, const igamg_options* opt,
                         void* cuda_stream, igamg_ctx** out);

/* Number of active (non-Dirichlet) dofs N_l of level l (-1 = finest). */
igamg_status igamg_num_dofs(const igamg_ctx* ctx, int level, int64_t* n);

/* Device memory the context holds (hierarchy, work vectors, graphs excluded), in bytes. */
igamg_status igamg_device_bytes(const igamg_ctx* ctx, int64_t* bytes);

/* Total number of patch-local basis functions sum_k prod_j n_kj at level l. */
igamg_status igamg_num_local(const igamg_ctx* ctx, int level, int64_t* n);

/* Host array local_to_global[sum_k prod_j n_kj]: for patch k (in order) and its local
 * tensor index (C order, last direction fastest) the global dof id, -1 if eliminated by a
 * Dirichlet side (Sec. 2 dof mapper). */
igamg_status igamg_dof_map(const igamg_ctx* ctx, int level, int64_t* local_to_global);

/* Physical coordinates of the Greville point of every active dof of level l (-1 =
 * finest): xyz[g*dim + a], host array of N_l * dim doubles.  The Greville abscissa of
 * B_i is (t_{i+1} + ... + t_{i+p}) / p per direction, mapped by the patch geometry G_k
 * (Sec. 2); a source f given as a function can be turned into spline coefficients
 * c_g = f(xyz_g) (Schoenberg's quasi-interpolant) for igamg_rhs_from_coefs. */
igamg_status igamg_greville_points(const igamg_ctx* ctx, int level, double* xyz);

/* Load vector b_i = (f_h, phi_i)_{L2(Omega)} of the source f_h = sum_j c_j phi_j given by
 * its spline coefficients c on the active dofs of the finest level (Sec. 2 right-hand side
 * (f, v)), by Gauss quadrature with the geometry.  Both device vectors of length N_L. */
igamg_status igamg_rhs_from_coefs(igamg_ctx* ctx, const double* coef_dev, double* rhs_dev);

/* PCG with one multigrid cycle (Algorithm 1) per iteration as preconditioner (Sec. 4),
 * started from x_dev (in: x_0, out: x), stopped when ||b - A x||_2 <= tol ||b - A x_0||_2
 * or after max_iter iterations (tol = 0 runs exactly max_iter).  Synchronises the stream.
 * `res` may be NULL. */
igamg_status igamg_solve(igamg_ctx* ctx, const double* rhs_dev, double* x_dev, double tol,
                         igamg_result* res);

/* Several right-hand sides of one problem solved together: igamg_solve for the nrhs device
 * vectors rhs_dev[q] (x_dev[q]: in x_0, out x; host arrays of nrhs device pointers, each
 * vector of length N_L, all distinct), each stopped by its own residual test.  Where the
 * problem qualifies (2D, every level above the coarsest of rectangle patches, V-cycle) the
 * lockstep engine of igamg_solve_batch runs them: each step of Algorithm 1 is one launch
 * over all right-hand sides, which share the hierarchy's constant arrays (1D factors,
 * smoother bases, transfer weights) and read them once per launch; the work arrays are
 * copied once per extra right-hand side on first use (kept until igamg_free, counted by the
 * context's device bytes).  This path runs the FP64 numerics whatever the precision option
 * (each answer meets the same tolerance); with a forced FD engine (fd_engine 1..4) and FP64
 * each answer is bit-identical to igamg_solve of that right-hand side alone.  Otherwise the
 * right-hand sides are solved one after the other by igamg_solve (also when the lockstep
 * engine cannot be built, e.g. without device memory for the copies).  `res` and `status` (may
 * be NULL) receive nrhs entries.  Returns the worst status (IGAMG_ERR_NOT_CONVERGED only if
 * nothing worse); IGAMG_ERR_ARG for nrhs < 1, null arrays or vectors, tol < 0.
 * Synchronises the stream. */
igamg_status igamg_solve_multi(igamg_ctx* ctx, int nrhs, const double* const* rhs_dev,
                               double* const* x_dev, double tol, igamg_result* res,
                               igamg_status* status);

/* igamg_solve with HOST vectors: copies rhs and x_0 to the device, solves, copies x back
 * (the end-to-end call).  Synchronises. */
igamg_status igamg_solve_host(igamg_ctx* ctx, const double* rhs_host, double* x_host,
                              double tol, igamg_result* res);

/* Single steps of the cycle, for per-step checks and measurement.  Device vectors in the
 * global numbering of the level named.
 *   igamg_apply:        y = A_l x                                  (Eq. linear:system)
 *   igamg_smooth:       z = L_l^{-1} r, l >= 1                      (Eq. additive)
 *   igamg_restrict:     rc = P_l^T r,  r on level l, rc on l-1, l >= 1  (Sec. 3)
 *   igamg_prolong:      u = P_l uc,    uc on level l-1, u on l, l >= 1  (Sec. 3)
 *   igamg_coarse_solve: x = A_0^{-1} r                             (Sec. 4, exact solve)
 *   igamg_precondition: z = Multigrid(L, 0, r)                      (Algorithm 1) */
igamg_status igamg_apply(igamg_ctx* ctx, int level, const double* x_dev, double* y_dev);
igamg_status igamg_smooth(igamg_ctx* ctx, int level, const double* r_dev, double* z_dev);
igamg_status igamg_restrict(igamg_ctx* ctx, int level, const double* r_dev, double* rc_dev);
igamg_status igamg_prolong(igamg_ctx* ctx, int level, const double* uc_dev, double* u_dev);
igamg_status igamg_coarse_solve(igamg_ctx* ctx, const double* r_dev, double* x_dev);
igamg_status igamg_precondition(igamg_ctx* ctx, const double* r_dev, double* z_dev);

/* Measurement of the cycle of Algorithm 1 as the solve runs it: z = Multigrid(L, 0, r) in
 * the context's working precision (FP64, or the FP32/BF16 inner cycle of the precision
 * variant, fed with r converted to FP32), captured once as a CUDA graph and replayed `reps`
 * times between CUDA events on the context's stream.  *ms = device time per cycle;
 * *bytes (may be NULL) = the algorithmic bytes of one cycle (band coefficients, vectors and
 * smoother bases read and written once, summed over the kernel classes of
 * igamg_profile_read).  Overwrites the context's cycle work vectors; synchronises. */
igamg_status igamg_cycle_time(igamg_ctx* ctx, const double* r_dev, int reps, double* ms, double* bytes);

/* Fast-diagonalisation apply of one tensor-product local smoother (Sec. 3: the
 * patch-interior subspace-corrected mass smoother in diagonalised form, L_T^{-1} =
 * (U0 x U1) diag(Dinv) (U0 x U1)^T), the core contraction of every smoothing step:
 *     Z = tau * U0 ((U0^T R U1) .* Dinv) U1^T.
 * No context needed.  Device pointers, FP64, row-major:
 *   U0 n0 x n0 and U1 n1 x n1 (columns = basis vectors), Dinv n0 x n1 (row stride n1),
 *   R n0 x n1 with row stride ldr >= n1, Z n0 x n1 with row stride ldz >= n1 (Z may be R
 *   itself when ldz == ldr: R is read completely before Z is written),
 *   scratch: caller-provided device buffer of 2*n0*n1 doubles, overwritten; it must not
 *   overlap any other argument.
 * Runs on `cuda_stream` (NULL = legacy default stream) and returns without synchronising.
 * Errors: IGAMG_ERR_ARG for n0, n1 < 1, ld < n1 or a NULL pointer (nothing is launched);
 * IGAMG_ERR_CUDA if a launch fails.  The message is available from igamg_last_error(NULL). */
igamg_status igamg_fd_apply(int n0, int n1, const double* U0, const double* U1, const double* Dinv,
                            const double* R, int ldr, double tau, double* Z, int ldz,
                            double* scratch, void* cuda_stream);

/* The same apply as igamg_fd_apply for callers that cannot allocate device memory: a
 * plugin or host framework that owns the device allocator and forbids allocations outside
 * it, a fixed-budget or real-time caller that may not allocate after start-up, or a
 * caller with no place to keep a scratch buffer between calls.  This entry point
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine); its scratch
 * is a fixed device array of 2 * 262144 doubles (4 MiB) built into the library, which
 * every GPU that loads the library holds until the process exits.  The paper has no
 * counterpart: this is a memory-management variant, not a step of the method.
 *   - Arguments and results are those of igamg_fd_apply without `scratch`.
 *   - n0 * n1 must not exceed 262144 (512 x 512); larger tiles are rejected with
 *     IGAMG_ERR_ARG and a message naming the limit, and nothing is launched.
 *   - Every call looks up the array's address on the current device (so a device reset
 *     between calls is harmless); the first call on a device also loads the library's
 *     device code there: make that first call before any stream capture.
 *   - All calls on a device share the one array, which keeps the last call's contents;
 *     every element is written before it is read, so nothing has to be cleared.  Calls
 *     whose kernels overlap on the GPU (different streams, or threads) race on the array:
 *     serialise them, e.g. on one stream.
 *   - Errors: IGAMG_ERR_ARG as above, IGAMG_ERR_CUDA if the lookup or a launch fails;
 *     message from igamg_last_error(NULL). */
igamg_status igamg_fd_apply_noalloc(int n0, int n1, const double* U0, const double* U1,
                                    const double* Dinv, const double* R, int ldr, double tau,
                                    double* Z, int ldz, void* cuda_stream);

/* Per-kernel-class accounting for measurement.  While enabled, the context counts every
 * kernel it launches; igamg_profile_read returns, for class `cls`, the launches, the summed
 * device time in ms, and the algorithmic FLOPs and bytes of those launches (the operands
 * the method itself must read and write once: band coefficients, vectors, smoother bases).
 * Classes: 0 stiffness apply/residual, 1 patch-interior smoother contractions, 2 interface
 * smoothers (gather, edge contractions, scatter), 3 transfers, 4 coarse solve, 5 vector
 * operations (reductions, PCG updates, conversions); class 6 counts no launches and holds in
 * `flops` the BF16 tensor-core FLOPs the tensor-core contractions execute (digit-slice
 * pairs and tile padding included; every tile of such a launch runs on the tensor cores);
 * class 7 is a sub-account of classes 1 and 2: the launches of the tensor-core contraction
 * kernel alone (their count, time and FP64 GEMM FLOPs).  `enable` is a bit mask of the
 * classes whose launches are bracketed by CUDA events on the launching stream (bit c =
 * class c; 0 disables); the
 * PCG iterations then replay a graph variant with event-record nodes (captured once per
 * mask).  Enabling resets the counters.  Reading synchronises the stream. */
igamg_status igamg_profile_enable(igamg_ctx* ctx, int enable);
igamg_status igamg_profile_read(igamg_ctx* ctx, int cls, int64_t* launches, double* ms,
                                double* flops, double* bytes);

/* FP64 throughput of the current device, the denominator of FP64 roofline fractions (not a
 * step of the method): kind 0 = FP64 FMA pipe (dependent FMA chains, 8 per thread), kind 1 =
 * FP64 tensor-core MMAs (mma.sync m8n8k4), `iters` iterations per chain over 4 blocks of
 * 256 threads per SM, timed with CUDA events after a warm-up.  *tflops = the rate;
 * *sm_count (may be NULL) = the device's multiprocessor count.  Synchronises the device. */
igamg_status igamg_micro_fp64(int kind, int64_t iters, double* tflops, int* sm_count);

/* Synchronises the context's stream. */
igamg_status igamg_sync(igamg_ctx* ctx);

/* Releases everything the context owns.  NULL-safe. */
igamg_status igamg_free(igamg_ctx* ctx);

/* Message of the last error on this context; with ctx == NULL, of the last failed setup
 * or context-free call on the calling thread.  Never NULL; valid until the next call. */
const char* igamg_last_error(const igamg_ctx* ctx);

/* ---------------------------------------------------------------- batched solves
 * Many independent problems (each the model problem of Sec. 2 on its own multi-patch
 * domain) solved together on one device.  Each problem keeps its own context: its
 * hierarchy stays resident between solves.  Two engines (igamg_options.batch_engine): the
 * lockstep engine runs PCG for all problems at once, each step of Algorithm 1 (apply,
 * smoother pieces, transfers, coarse solves) one launch over the tiles of every problem at
 * that depth below its finest level, each PCG iteration of the whole batch one CUDA graph
 * replay; the worker-stream engine runs whole single solves on `workers` host threads with
 * a CUDA stream each, in decreasing order of estimated work.  With worker streams, or with a
 * forced FD engine (fd_engine 1..4), a problem's result is bit-identical to igamg_solve on
 * that problem alone; with the autotuned default the lockstep engine runs every level whose
 * tensor-core stages exist on the tensor cores (its launches hold the tiles of all problems),
 * which can differ from a problem's own choice by FP64 rounding.  The paper solves one
 * problem at a time and has no counterpart of this layer. */
typedef struct igamg_batch igamg_batch;

/* Sets up `count` problems (host array, read during the call) with the same options.
 * workers <= 0 selects 16 (capped at count).  The contexts use `cuda_stream` outside
 * igamg_solve_batch.  On failure nothing is kept and igamg_last_error(NULL) names the first
 * failing problem. */
igamg_status igamg_setup_batch(const igamg_problem* problems, int count, const igamg_options* opt, int workers,
                               void* cuda_stream, igamg_batch** out);

/* The context of problem i (owned by the batch; do not free): for igamg_num_dofs,
 * igamg_dof_map, igamg_rhs_from_coefs, igamg_solve and the other per-context calls. */
igamg_status igamg_batch_context(igamg_batch* batch, int i, igamg_ctx** ctx);

/* Solves problem i for rhs[i] into x[i] (host arrays of `count` device pointers, each of
 * that problem's igamg_num_dofs; x[i] holds the initial guess on entry), every problem to
 * the relative tolerance tol.  Starts after the work queued on the batch's stream and
 * returns when every solve is done.  res and status (host arrays of `count`, or NULL)
 * receive each problem's result and status.  Returns IGAMG_OK if every solve converged,
 * else the first other status by problem index, an error taking precedence over
 * IGAMG_ERR_NOT_CONVERGED. */
igamg_status igamg_solve_batch(igamg_batch* batch, const double* const* rhs, double* const* x, double tol,
                               igamg_result* res, igamg_status* status);

/* The engine igamg_solve_batch uses: *engine = 0 lockstep (every step of the cycle one
 * launch over all problems), 1 worker streams.  For the lockstep engine, the kernel launches
 * of the last igamg_solve_batch, their algorithmic FLOPs (the FP64 operations of the
 * method) and the BF16 tensor-core FLOPs of its FD contractions; -1 for worker streams.
 * launches, flops and mma_flops may be NULL. */
igamg_status igamg_batch_engine(igamg_batch* batch, int* engine, int64_t* launches, double* flops,
                                double* mma_flops);

/* Releases every context of the batch and its streams.  NULL is accepted. */
igamg_status igamg_free_batch(igamg_batch* batch);

/* ---------------------------------------------------------------- serving
 * A request is one right-hand side of a registered model (a problem as in igamg_setup).
 * Requests are answered by `workers` host threads with a CUDA stream each, in arrival
 * order, except that a request waits while another worker uses its model's hierarchy.
 * A worker that takes a request of a model igamg_solve_multi runs in lockstep also takes
 * the model's other waiting requests of the same tolerance (oldest first, up to 16 in all)
 * and solves them together with igamg_solve_multi (one launch per step for the group, the
 * hierarchy's constant arrays shared; FP64 numerics); other models' requests are solved
 * one at a time with igamg_solve.
 * Hierarchies stay resident between requests; a model's hierarchy is built on its first
 * request when its estimated size fits the device-memory budget, after freeing the least
 * recently used idle hierarchies.  Times are milliseconds since igamg_server_create.  The
 * paper solves one problem at a time and has no counterpart of this layer. */
typedef struct igamg_server igamg_server;

typedef struct {
  int status;           /* igamg_status of the solve (IGAMG_ERR_OOM: the model never fits) */
  int iters;            /* PCG iterations */
  double relres;        /* ||b - A x|| / ||b|| at exit                                 */
  double t_submit_ms;   /* igamg_server_submit                                       */
  double t_start_ms;    /* a worker took the request                                 */
  double t_done_ms;     /* solution copied to x                                      */
  double setup_ms;      /* hierarchy built for this request (0 if it was resident)    */
  int group;            /* requests solved together with this one, itself included   */
} igamg_request_info;

typedef struct {
  int models, resident;
  int64_t device_bytes;  /* hierarchies (measured; estimates while being built)        */
  int64_t setups, evictions, completed, waiting;
  int64_t groups;        /* igamg_solve_multi calls of more than one request          */
  int64_t grouped;       /* requests answered by those calls                          */
} igamg_server_counters;

/* Starts the workers.  opt (NULL = defaults) applies to every model; hbm_budget_bytes
 * bounds the device memory of the resident hierarchies. */
igamg_status igamg_server_create(const igamg_options* opt, int workers, int64_t hbm_budget_bytes,
                                 igamg_server** out);

/* Registers a problem (copied; nothing is built yet) and returns its model id, the length
 * of its right-hand side and solution (the library's dof order of igamg_dof_map) and the
 * estimated device bytes of its hierarchy used for admission until it is first built
 * (num_dofs and est_bytes may be NULL). */
igamg_status igamg_server_add_model(igamg_server* server, const igamg_problem* problem, int* model,
                                    int64_t* num_dofs, int64_t* est_bytes);

/* Queues a solve of model `model` for the load vector rhs (host, num_dofs values) from
 * x = 0 to the relative tolerance tol; the solution is written to x (host).  Both arrays
 * must stay valid until igamg_server_wait returns for the request. */
igamg_status igamg_server_submit(igamg_server* server, int model, const double* rhs, double* x, double tol,
                                 int64_t* request);

/* Blocks until the request is answered and returns its record (each request is waited
 * for exactly once). */
igamg_status igamg_server_wait(igamg_server* server, int64_t request, igamg_request_info* info);

igamg_status igamg_server_stats(igamg_server* server, igamg_server_counters* stats);

/* Stops the workers (after the requests they are running) and frees every hierarchy.
 * Requests still queued are dropped: wait for them first.  NULL is accepted. */
igamg_status igamg_server_free(igamg_server* server);

#ifdef __cplusplus
}
#endif

#endif /* IGAMG_H */
