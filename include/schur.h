/*
 * libschur — GB300 (sm_103a) solver for the negative Schur complement of distributed optimal
 * control with a Poisson constraint, applied through its exact complex factorisation.
 *
 * Problem (arXiv 1312.5653, Sec. 2): uniform Q1 elements on the unit box [0,1]^d (d = 2 or 3),
 * nel[a] elements along axis a, homogeneous Dirichlet conditions on the whole boundary.  K is the
 * stiffness and M the consistent mass (the paper's volume matrix V) on the n = prod(nel[a]-1)
 * interior nodes.  Vectors are real FP64, one entry per interior node, lexicographic with axis 0
 * fastest; several right-hand sides are stored column-major with leading dimension ld >= n.
 * beta is the paper's regularisation phi, gamma = 1/sqrt(beta).
 *
 *   S = K M^{-1} K + M / beta                                   (Sec. 3.1, Schur complement)
 *   S = (K + i gamma M) M^{-1} (K - i gamma M)                  (Sec. 4, exact factorisation)
 *   S^{-1} b = -Im(z) / gamma,  z = (K + i gamma M)^{-1} b      (b real; follows from Sec. 4:
 *            A - conj(A) = 2 i gamma M, so S^{-1} = (conj(A)^{-1} - A^{-1}) / (2 i gamma))
 *
 * The complex-symmetric factor A = K + i gamma M is solved by a FETI-DP dual iteration (Sec. 5):
 * non-overlapping subdomains (nsub[a] per axis), primal subdomain corners with a coarse problem,
 * GMRES on the interface multipliers with the Dirichlet preconditioner, per-subdomain complex
 * LDL^T factors.  Optional mixed precision runs the FETI-DP solve in complex FP32 and refines
 * z in FP64 on the residual b - A z (Sec. 3.1 names iterative refinement in higher precision
 * as the remedy for the accuracy loss of the range-space method).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers owned by the caller (never freed by the library);
 *     *_host are host pointers (pageable or pinned).
 *   - Work is ordered on the CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Calls return after enqueueing unless the description says they synchronise.
 *   - Return value: SCHUR_OK (0) or a negative SCHUR_E* code; no C++ exception crosses the ABI.
 *     schur_last_error() gives a message for the calling thread's most recent failure.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef SCHUR_H
#define SCHUR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCHUR_OK 0
#define SCHUR_EINVAL -1     /* bad argument (mesh, beta, sizes, pointers)                      */
#define SCHUR_ENOMEM -2     /* device or host allocation failed                                */
#define SCHUR_ENOTCONV -3   /* tolerance not met within max_iter / max_refine; x still written */
#define SCHUR_EBREAKDOWN -4 /* zero or non-finite pivot / Krylov breakdown / non-finite data    */
#define SCHUR_ETIMEOUT -5   /* a bounded device or host wait gave up                           */
#define SCHUR_ECUDA -6      /* a CUDA runtime call failed                                      */
#define SCHUR_EBUSY -7      /* serving: admission refused (memory budget or queue full)        */

#define SCHUR_FP64 0   /* FETI-DP solve in complex FP64                                         */
#define SCHUR_MIXED 1  /* FETI-DP solve in complex FP32, FP64 refinement of z on b - A z        */

#define SCHUR_LOCAL_PER_SUBDOMAIN 0 /* one factor and one set of local operators per subdomain  */
#define SCHUR_LOCAL_SHARED 1        /* subdomains with identical local matrices share them      */

#define SCHUR_FACTOR_EXACT 0 /* S_c = (K + i gamma M) M^{-1} (K - i gamma M) = S exactly (Sec. 4)     */
#define SCHUR_FACTOR_PW 1    /* S_p = (K + gamma M) M^{-1} (K + gamma M) = S + 2 gamma K, the
                                Pearson-Wathen approximation (Sec. 3.2, Eq. pearsonapproximation)     */

typedef struct schur_ctx schur_ctx;

typedef struct {
  int dim;    /* 2 or 3 */
  int nel[3]; /* elements per axis (entries beyond dim ignored) */
} schur_mesh;

typedef struct {
  int nsub[3];       /* subdomains per axis; nel[a] % nsub[a] == 0, nel[a]/nsub[a] >= 2   */
  int precision;     /* SCHUR_FP64 or SCHUR_MIXED                                         */
  double tol;        /* outer stop: ||b - A z||_2 / ||b||_2 <= tol for every right-hand side */
  double inner_tol;  /* GMRES stop: dual residual / initial dual residual (<= 0: default)  */
  int max_iter;      /* GMRES iterations per inner solve (Krylov basis size, no restart)  */
  int max_refine;    /* outer refinement steps (each one inner FETI-DP solve)             */
  int local_mode;    /* SCHUR_LOCAL_PER_SUBDOMAIN or SCHUR_LOCAL_SHARED                   */
  int tc_split;      /* mixed 3D local operators on the tensor cores (TF32 inputs, FP32
                        accumulation): 0 or 3 = three products hi*hi + hi*lo + lo*hi of the
                        split x = hi + lo (FP32 accuracy), 1 = one product (TF32 rounding)     */
  int factor;        /* which Schur complement schur_solve inverts: SCHUR_FACTOR_EXACT (S, by one
                        complex FETI-DP solve with K + i gamma M and x = -Im(z)/gamma) or
                        SCHUR_FACTOR_PW (S_p, by two real FETI-DP solves with K + gamma M and
                        one M product: x = (K + gamma M)^{-1} M (K + gamma M)^{-1} b)          */
  int augment;       /* 1: augmented coarse problem (Sec. 5): besides the corners, one coarse
                        unknown per pair of face-adjacent subdomains enforcing a zero average
                        jump across that face at every iteration (the translational edge mode
                        of the paper's RAUG; a face in 3D); the coarse matrix is inverted
                        densely in FP64, so at most 4096 coarse unknowns (EINVAL beyond)      */
  int reserved[2];   /* must be zero                                                      */
} schur_opts;

typedef struct {
  int status;          /* the return code of the call that filled it                      */
  int outer_steps;     /* refinement steps taken                                           */
  int iters_total;     /* GMRES iterations summed over steps (max over right-hand sides)   */
  int iters_first;     /* GMRES iterations of the first step                               */
  double rel_residual; /* final ||b - A z|| / ||b||, max over right-hand sides (FP64)       */
  double ms_setup;     /* schur_setup wall time (host clock, includes device sync)         */
  double ms_solve;     /* this call's wall time, when the call synchronises; else 0        */
} schur_stats;

typedef struct {
  long long n;         /* interior dofs                                                    */
  int n_sub;           /* subdomains                                                       */
  int n_classes;       /* distinct local operator sets stored                              */
  int n_lambda;        /* dual unknowns (interface multipliers)                            */
  int n_coarse;        /* primal corner unknowns                                           */
  int n_delta;         /* interface slots per subdomain                                    */
  int n_local;         /* nodes per subdomain grid ((s+1)^d)                               */
  long long bytes_operators; /* device bytes held by factors and local/coarse operators     */
} schur_info_t;

/* Defaults: nsub = 4 per axis, FP64, tol 1e-12, inner_tol by precision (1e-12 FP64, 3e-5
 * mixed), max_iter 300, max_refine 8, per-subdomain local operators, tc_split 0 (three TF32
 * products). */
void schur_default_opts(schur_opts* opts);

/* Builds the solver for one mesh and beta: per-subdomain Q1 assembly of K + i gamma M, batched
 * complex LDL^T (no pivoting; the real and imaginary parts are positive definite) of the
 * remainder matrices A_rr (subdomain nodes minus corners and Dirichlet nodes, Sec. 5) and of the
 * interior matrices A_ii, the explicit local dual operators B A_rr^{-1} B^T, the corner coupling,
 * the Dirichlet-preconditioner Schur complements S_bb (Eq. WS), and the coarse corner problem
 * (factorised in FP64).  Synchronises `stream` before returning.  *out receives the context.
 * Errors: EINVAL (mesh/beta/opts), ENOMEM, EBREAKDOWN (zero pivot), ECUDA. */
int schur_setup(const schur_mesh* mesh, double beta, const schur_opts* opts, void* stream,
                schur_ctx** out);

/* x = S^{-1} b for nrhs right-hand sides (Sec. 3.1, Eq. schurcomplementsystem with b given):
 * one complex FETI-DP solve per refinement step, then x = -Im(z)/gamma.  With b = M y_bar the
 * result is x = beta y* (state of the KKT system of Sec. 2); with b = K y_bar it is lambda*.
 * b_dev, x_dev: device FP64, n x nrhs, leading dimension ld.  Synchronises `stream` (the host
 * reads convergence flags).  Returns ENOTCONV with x written if the tolerance is not met.
 * st may be NULL.  nrhs == 0 is a no-op. */
int schur_solve(schur_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int ld, void* stream,
                schur_stats* st);

/* As schur_solve with host buffers: copies b to the device, solves, copies x back, all on
 * `stream`; synchronises before returning. */
int schur_solve_host(schur_ctx* ctx, const double* b_host, double* x_host, int nrhs, int ld,
                     void* stream, schur_stats* st);

/* z = A^{-1} (b_re + i b_im) with the context's factor A: K + i gamma M (one factor of Sec. 4, the
 * factor the shortcut uses) or, with SCHUR_FACTOR_PW, the real K + gamma M of S_p (Sec. 3.2).
 * b_im_dev may be NULL (real right-hand side).  z_dev: interleaved complex FP64 (re, im), n x nrhs
 * with leading dimension ld complex entries.  Synchronises.  Same refinement and stop rule as
 * schur_solve. */
int schur_complex_solve(schur_ctx* ctx, const double* b_re_dev, const double* b_im_dev, double* z_dev,
                        int nrhs, int ld, void* stream, schur_stats* st);

/* y = M x and y = K x (FP64 matrix-free Q1 stencils).  Asynchronous. */
int schur_apply_mass(schur_ctx* ctx, const double* x_dev, double* y_dev, int nrhs, int ld, void* stream);
int schur_apply_stiffness(schur_ctx* ctx, const double* x_dev, double* y_dev, int nrhs, int ld,
                          void* stream);

/* y = S x = K M^{-1} K x + M x / beta in FP64 (Sec. 3.1, Eq. schurcomplementsystem); K and M are
 * matrix-free Q1 stencils, M^{-1} is a fixed-degree Chebyshev iteration with Jacobi scaling on the
 * Q1 mass spectrum bounds lambda(D^{-1} M) in (2^-d, (3/2)^d), the degree chosen for a relative
 * error of 1e-15 (a fixed linear operator).  Not on the solve path (used by the refinement tests and
 * by callers that need S itself).  x_dev, y_dev: n x nrhs, leading dimension ld >= n; only the
 * first n entries of each column are read or written.  Synchronises.  Errors: EINVAL, ENOMEM
 * (first call with more columns than before grows the context's workspace), ECUDA. */
int schur_apply_S(schur_ctx* ctx, const double* x_dev, double* y_dev, int nrhs, int ld, void* stream);

/* y = S x as schur_apply_S, but with no context and no device allocation at all (the paper has no
 * counterpart; this is a deployment convenience).  For callers that cannot allocate device
 * memory: code that runs where cudaMalloc is unavailable or not allowed, such as a plugin inside
 * another runtime's stream-ordered region or a process whose allocator is owned by its host
 * application, and that therefore cannot call schur_setup.  The work vectors live in one fixed
 * device array of 5 x 2^20 doubles (40 MiB) that every GPU loading the library holds until the
 * process exits, so n (interior nodes of the mesh) must be at most 2^20; larger meshes return
 * SCHUR_EINVAL.  Columns are processed one after another (any nrhs; ld >= n).
 * The first call on a device looks up the array's device address with that device current; make
 * that first call before any stream capture.  All calls on all streams share the one array and
 * every call overwrites it completely before reading it: calls whose work overlaps on the GPU race
 * and must be ordered by the caller.  x_dev and y_dev must not overlap (EINVAL).  Asynchronous on
 * `stream`.  Errors: EINVAL (with a message in schur_last_error), ECUDA. */
int schur_apply_S_static(const schur_mesh* mesh, double beta, const double* x_dev, double* y_dev, int nrhs, int ld,
                         void* stream);

/* The range-space method of Sec. 3.1 with Dirichlet data y = y_c on the boundary (the thermal
 * problem of Sec. 6.1, Eqs. heatconduction and ex1boundarycondition: y_c = ybar there).
 * ybar_full_dev: the target state on all prod(nel[a] + 1) grid nodes, boundary included
 * (lexicographic, axis 0 fastest, leading dimension ldf); its boundary values are taken as y_c.
 * Computes, on the n interior nodes (leading dimension ld >= n):
 *   lambda = S^{-1} (K ybar + K_c y_c)            (Eq. schurcomplementsystem, by schur_solve)
 *   y = ybar - M^{-1} K lambda,  u = lambda / beta (Eq. updateyandu; M^{-1} as in schur_apply_S)
 * and, when viol_host != NULL, viol_host[c] = ||K y + K_c y_c - M u||_2 / ||K y||_2 for every
 * column (the relative constraint violation, Eq. relativeconstraintviolation).  lambda_dev may be
 * NULL.  Needs a context with factor SCHUR_FACTOR_EXACT.  Synchronises.  Returns ENOTCONV (outputs
 * written) if the S solve misses its tolerance; EINVAL, ENOMEM, ECUDA as schur_solve. */
int schur_control_solve(schur_ctx* ctx, const double* ybar_full_dev, int ldf, double* y_dev, double* u_dev,
                        double* lambda_dev, int nrhs, int ld, double* viol_host, void* stream, schur_stats* st);

/* Full-space KKT system of Sec. 2 with homogeneous Dirichlet data:
 *   [M 0 K; 0 beta M -M; K -M 0] (y, u, l).
 * Vectors hold the three blocks stacked: entries [0,n) = y, [n,2n) = u, [2n,3n) = lambda; ld >= 3n.
 * schur_kkt_apply: r = KKT v (asynchronous).
 * schur_kkt_precond_apply: z = P_mgw^{-1} r with P_mgw = diag(M, beta M, S) (Sec. 3.2,
 *   Eq. murphypreconditioner): M^{-1} by Chebyshev iteration with Jacobi scaling on the Q1 mass
 *   spectrum bounds (fixed degree, a fixed linear operator), S^{-1} by schur_solve.  With the
 *   factor SCHUR_FACTOR_PW the third block is S_p^{-1} (the Pearson-Wathen approximation of
 *   Eq. pearsonapproximation in place of S).  Synchronises.
 * schur_kkt_minres: MINRES on the KKT system preconditioned by P_mgw, FP64 Krylov, stop at
 *   ||r_k||/||r_0|| <= tol (preconditioned norm); iters receives the iteration count (max over
 *   right-hand sides).  Synchronises.  ENOTCONV if max_it is reached. */
int schur_kkt_apply(schur_ctx* ctx, const double* v_dev, double* r_dev, int nrhs, int ld, void* stream);
int schur_kkt_precond_apply(schur_ctx* ctx, const double* r_dev, double* z_dev, int nrhs, int ld,
                            void* stream);
int schur_kkt_minres(schur_ctx* ctx, const double* rhs_dev, double* sol_dev, int nrhs, int ld, double tol,
                     int max_it, int* iters, void* stream);

/* Host-only (no GPU needed): the FETI-DP partition of Sec. 5 for a mesh and nsub.
 * schur_partition fills info (bytes_operators = 0) without touching the device.
 * schur_partition_export copies one index map into out (int32, capacity cap entries):
 *   which = 0: lambda sides, 2 per multiplier: subdomain*n_delta + slot (+1 side, then -1 side)
 *           1: interface slot -> local node index                        (n_delta)
 *           2: subdomain corner -> coarse unknown or -1, 2^dim per subdomain
 *           3: subdomain -> operator class                               (n_sub)
 * Returns EINVAL for a bad mesh/nsub or a too small buffer. */
int schur_partition(const schur_mesh* mesh, const int* nsub, int local_mode, schur_info_t* info);
int schur_partition_export(const schur_mesh* mesh, const int* nsub, int local_mode, int which, int* out,
                           long long cap);

/* Kernel timing for measurement (not needed to solve).  schur_profile_begin enables, for every
 * category whose bit is set in mask, a CUDA event pair recorded on the launching stream around
 * each launch.  schur_profile_end synchronises the device, writes per-category launch counts and
 * summed event times (ms) into out (up to cap entries; *count = categories seen) and disables
 * timing.  Categories: 0 factor, 1 form, 2 coarse_setup, 3 local_rhs, 4 apply_F, 5 apply_S,
 * 6 scatter, 7 coarse_apply, 8 corner, 9 gmres_dots, 10 gmres_update, 11 gmres_other,
 * 12 recover, 13 assemble_z, 14 residual, 15 coarse_inverse, 16 interior, 17 form_corner (the
 * corner columns of the local operators, formed ahead of F on the 2D corner coarse problem).
 * schur_launch_count: kernels launched through ctx since schur_setup (setup included). */
typedef struct {
  int category;
  long long launches;
  double total_ms;
} schur_kernel_time;
int schur_profile_begin(unsigned mask);
int schur_profile_end(schur_kernel_time* out, int cap, int* count);
const char* schur_kernel_category_name(int category);
long long schur_launch_count(const schur_ctx* ctx);

/* Arithmetic peak probe (measurement aid, no paper counterpart): runs one in-register or
 * in-shared-memory loop of `iters` iterations on every SM of the current device, once to warm up
 * and once timed with CUDA events on `stream`, and writes the achieved TFLOP/s to *tflops.
 * kind 0: FP64 FMA (CUDA cores); 1: FP32 FMA (CUDA cores); 2: FP64 tensor MMA (mma.sync
 * m8n8k4); 3: TF32 tensor MMA (tcgen05.mma kind::tf32, 128 x 256 x 8, accumulator in tensor
 * memory).  These are the denominators of the ALU and tensor-pipe rooflines reported for this
 * library's kernels.  Allocates a small output buffer; synchronises.  Errors: EINVAL,
 * ETIMEOUT (tensor-core completion wait gave up), ECUDA. */
int schur_peak_probe(int kind, int iters, double* tflops, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Serving.  A server owns worker threads (one CUDA stream each, on the device current at
 * creation) and a device-resident cache of contexts keyed by (mesh, beta) with the server's
 * precision, evicted least-recently-used when a new context would exceed device_mem_budget.
 * Subdomains are 16 elements per side in 2D and 8 in 3D (or the nearest divisor of nel).
 * schur_submit queues a request (host buffers b, x of n x nrhs, column-major, ld = n; both must
 * stay valid until the request completes).  A request is admitted when its context is cached or
 * memory for a new one can be freed; queued requests with the same (mesh, beta) are solved
 * together as one multi-RHS solve of up to max_batch_rhs columns (requests arriving while other
 * work runs join the next batch of their key); batches of different keys run concurrently on the
 * worker streams.  Results equal those of separate schur_solve calls within the solver
 * tolerance (each column is refined until every column of the batch meets tol).
 * schur_poll: 0 done (st filled; st->ms_solve = submit-to-completion latency in ms), 1 pending,
 * <0 the request's error.  schur_wait: the same after waiting at most timeout_ms
 * (SCHUR_ETIMEOUT if still pending).  schur_submit returns SCHUR_EBUSY when the request can never
 * fit the budget.  No paper counterpart (Sec. 4 notes that multiple right-hand sides favour reusing
 * factorisations). */
typedef struct schur_server schur_server;
typedef struct {
  size_t device_mem_budget; /* bytes of device memory the cache and workspaces may hold        */
  int workers;              /* worker threads / streams (concurrent batches)                   */
  int precision;            /* SCHUR_FP64 or SCHUR_MIXED                                       */
  double tol;               /* outer tolerance of every solve                                  */
  int max_batch_rhs;        /* columns per batched solve                                       */
  int max_iter;             /* GMRES iterations per inner solve                                */
  int reserved[4];
} schur_server_opts;
typedef struct {
  int cached_contexts, queued;
  long long completed, bytes_reserved;
  long long batches;         /* multi-RHS solves run (one per batch)                              */
  long long batch_columns;   /* right-hand sides summed over those solves                         */
  long long shared_requests; /* requests solved in one batch together with at least one other     */
  long long setups;          /* contexts built (factor-cache misses)                              */
  int max_concurrent;        /* most batches running on the device at the same time               */
  int reserved[3];
} schur_server_info_t;
void schur_server_default_opts(schur_server_opts* opts);
int schur_server_create(const schur_server_opts* opts, schur_server** out);
int schur_submit(schur_server* srv, const schur_mesh* mesh, double beta, const double* b_host, int nrhs,
                 double* x_host, long long* ticket);
int schur_poll(schur_server* srv, long long ticket, schur_stats* st);
int schur_wait(schur_server* srv, long long ticket, double timeout_ms, schur_stats* st);
int schur_server_info(schur_server* srv, schur_server_info_t* info);
void schur_server_destroy(schur_server* srv);

int schur_get_info(const schur_ctx* ctx, schur_info_t* info);
long long schur_ndof(const schur_mesh* mesh);
void schur_destroy(schur_ctx* ctx);
const char* schur_strerror(int code);
const char* schur_last_error(void);

/* Test hook: copies one local operator of class `cls` to host memory as interleaved complex FP64.
 * which = 0: F  = (A_rr^{-1}) restricted to the interface slots      (n_delta x n_delta)
 *         1: Frc = (A_rr^{-1} A_rc) on the interface slots           (n_delta x 2^d)
 *         2: S_bb = A_DD - A_Di A_ii^{-1} A_iD (Dirichlet precond.)  (n_delta x n_delta)
 *         3: the assembled coarse matrix, dense (corner-only coarse)  (n_coarse x n_coarse)
 *         4: the coarse inverse actually applied                     (n_coarse x n_coarse)
 *         5: the coupling columns [Frc | F Q] of the augmented coarse problem
 *            (n_delta x (2^d + 2d); without augmentation Frc alone)
 *         6: the layer pivot inverses D_K^{-1} of the block LDL^T factorisation of the class's
 *            remainder matrix on the full local grid of (s+1)^d nodes (layers along the last axis,
 *            L = s+1 blocks of b = (s+1)^(d-1) nodes; removed nodes are identity rows)  (L x b x b)
 * Row-major.  `cap` = capacity of out in complex entries.  Synchronises. */
int schur_debug_operator(schur_ctx* ctx, int which, int cls, double* out_host, long long cap);

#ifdef __cplusplus
}
#endif
#endif
