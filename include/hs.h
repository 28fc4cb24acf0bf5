/*
 * hs.h -- C ABI of the GB300 moving-PML sweeping preconditioner library (libhs.so).
 *
 * The library solves the 2D PML-stretched Helmholtz equation discretised by
 * the 5-point scheme of Engquist & Ying (2010), Sec. 2.1, Eq. helmd:
 *
 *   Delta u + omega^2 / c^2(x) u = f   on (0,1)^2, PML on all four sides,
 *
 * on the grid p_ij = (ih, jh), h = 1/(n+1), 1 <= i, j <= n, preconditioned by
 * the approximate sweeping factorisation with moving PMLs (Sec. 2.2-2.3,
 * Algorithms 3 and 4, two fronts, d layers per step).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Vectors.  Complex, interleaved (re, im).  One right-hand side (RHS) is a
 *   contiguous n*n array in the paper's ordering (x1 fastest, row by row in
 *   x2, Sec. 2.1); RHS r starts at element r*n*n.  dtype HS_C64 means
 *   float2 elements, HS_C128 double2 elements.
 * Pointers.  Vector pointers are DEVICE pointers unless stated otherwise; the
 *   caller owns them.  The plan owns every factor and workspace buffer.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All work of a call is enqueued on that stream; calls return
 *   after enqueueing except where stated.
 * Errors.  Every entry point returns an hs_status.  Asynchronous device
 *   errors (pivot breakdown, expired bounded waits) are recorded in a status
 *   word of the plan and reported by the next synchronising call
 *   (hs_solve, hs_sync) or by hs_last_device_status().  Nothing throws.
 */
#ifndef HS_H_
#define HS_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HS_OK = 0,
  HS_EINVAL = 1,       /* invalid argument: even n, widths too large, NULL pointer, nrhs out of range */
  HS_ENOMEM = 2,       /* device allocation failed */
  HS_EBREAKDOWN = 3,   /* zero pivot while inverting a diagonal block of a subproblem factor */
  HS_ETIMEOUT = 4,     /* a bounded device-side wait (TMA barrier) expired */
  HS_ENOCONV = 5,      /* FGMRES did not reach the tolerance within maxit, or produced NaN */
  HS_ECUDA = 6,        /* CUDA runtime error */
  HS_EUNSUPPORTED = 7  /* configuration outside what the kernels are built for */
} hs_status;

enum { HS_C64 = 64, HS_C128 = 128 };

/* Tuning and method constants.  hs_default_options() fills the defaults. */
typedef struct {
  double alpha;          /* alpha of Eq. helmalpha: the subproblems use (omega + i alpha)^2 / c^2.   default 2 */
  double pml_C;          /* C of Eq. sigma: strength of the boundary PML (part of the operator A).    default 20 */
  double moving_pml_C;   /* strength of the moving PMLs of the subproblems (Eq. helma).  0: the
                            boundary PML's pml_C, the single constant C that Eq. helma reuses
                            through sigma_2 (the paper's preconditioner); > 0: a separate
                            strength, a tuning of the preconditioner only (the operator A and
                            its solution do not change).                                      default 0 */
  int layers_per_step;   /* d of Sec. 2.3 (rows eliminated per sweep step).                           default 12 */
  int factor_prec;       /* HS_C64: complex float factors and sweep; HS_C128: complex double.          default HS_C64 */
  int chunk;             /* x1 columns per partition chunk (>= 2).  0: ceil(n / (SMs/2)), one chunk
                            CTA per SM pair and front (a full wave); any length is raised until the
                            separator count fits the separator solve's shared memory.        default 0 */
  int max_nrhs;          /* largest nrhs any later call will use (workspace is sized at setup).       default 64 */
  int restart;           /* FGMRES restart length m.                                                  default 20 */
  int reorth;            /* 0: classical Gram-Schmidt; 1: CGS with a second pass when needed (DGKS).  default 0 */
  long long spin_budget; /* SM clock cycles a device-side barrier wait may take before HS_ETIMEOUT.   default 1<<30 */
  int graphs;            /* 1: hs_apply replays the stage chain of the sweep as a CUDA graph
                            (captured on first use per nrhs); 0: direct launches.  hs_solve on a
                            2D plan sweeps a different Krylov vector at every step and launches
                            directly; on a 3D plan it replays the graph on the plan's own vector
                            and copies the result out.                                      default 1 */
  int krylov_basis;      /* 2D complex64 plans: 0 FGMRES with a double-float Arnoldi basis; 1 mixed-
                            precision refinement: cycles of FGMRES with an FP32 basis (FP32
                            products A z_j and Gram-Schmidt) restarted from the double-float
                            true residual, x updated in double-float (a network attached with
                            hs_attach_cnn uses mode 0).                                      default 1 */
  double inner_tol;      /* refinement cycles end when their residual estimate has fallen by this
                            factor (or below tol).                                             default 1e-4 */
  int frontal_gemm;      /* 3D setup, frontal Schur updates of complex64 factors (Sec. 4.2): 0 CUDA-
                            core FP32 FMA; tensor cores with FP32 accumulation: 1 TF32 (one pass),
                            3 3xTF32 (split operands, FP32-level accuracy), 2 BF16 (one pass),
                            4 3xBF16 (split operands, about 16 significant bits).  The blocked
                            inverse of large front pivot blocks uses the split form of the same
                            operand type.  Complex128 factors use FP64 FMA.                   default 3 */
  const char* tune_cache;/* path of the table written by hs_autotune; with chunk = 0, hs_setup
                            takes the chunk length (and, with sep_rhs_per_cta = 0, the separator
                            grouping) from it when it holds the problem's key.  NULL: not used.
                            The string must outlive the hs_setup call.                        default NULL */
  int sep_rhs_per_cta;   /* RHS per CTA of the separator solve (phase 2 of every sweep stage):
                            0 picks one while the RHS of both fronts fit on the SMs one CTA each,
                            else two or four; 1, 2 or 4 fix it (complex128 factors: at most two). default 0 */
  int two_front;         /* 1: PML on all four sides, two fronts sweeping toward the middle layer
                            (Sec. 2.3, every experiment of the paper).  0 (2D only): the formulation
                            of Sec. 2.1-2.2 and Algorithms 3-4 as printed: zero Dirichlet values at
                            x2 = 1, the one-sided sigma_2 of Eq. sigma at x2 = 0, one upward sweep
                            from the front F; the operator A changes accordingly (hs_matvec and
                            hs_solve use it), and n may be even.                        default 1 */
  int buffer_rows;       /* k >= 0 rows between each block and its moving PML (Sec. 2.2, the
                            buffer layers): window [lo - k - b + 1, hi] (mirrored for the upper
                            front, both sides for the middle layer).  A window that would cross
                            the grid boundary is cut there and keeps the operator's own profile
                            (the exact Schur inverse).  2D only; windows must stay <= 32 rows.
                                                                                           default 0 */
  int async_setup;       /* 1 (2D hs_setup only): hs_setup returns as soon as the factorisation is
                            queued on its stream instead of waiting for it, so that the caller can
                            overlap its own work (e.g. uploading right-hand sides) with the setup
                            kernels.  Every later call on the plan orders itself after the setup
                            on its own stream; a zero pivot is then reported by the next call that
                            synchronises (hs_sync, hs_solve, hs_last_device_status) instead of by
                            hs_setup.  The velocities are copied before hs_setup returns either
                            way.  No counterpart in the paper.                          default 0 */
} hs_options;

typedef struct hs_plan hs_plan;

/* Per-solve report, filled by hs_solve (host memory owned by the caller). */
typedef struct {
  int iterations;        /* FGMRES iterations (Arnoldi steps) until the last RHS converged */
  int restarts;          /* restart cycles started */
  int applies;           /* preconditioner applications (each over all nrhs) */
  double max_relres;     /* max over RHS of the final FP64 true relative residual ||f - A u|| / ||f|| */
  double t_apply_ms;     /* device time spent in M_alpha applications */
  double t_matvec_ms;    /* device time in A z products */
  double t_orth_ms;      /* device time in Gram-Schmidt and updates */
  double t_total_ms;     /* wall time of the call */
  int cnn_applies;       /* (direction, RHS) pairs for which the judge kept the network's correction */
} hs_solve_info;

/* Fill *opt with the defaults listed above.  Returns HS_EINVAL if opt is NULL. */
int hs_default_options(hs_options* opt);

/*
 * hs_setup -- build the sweeping factorisation (Algorithm 3, Sec. 2.3).
 *
 * c        HOST pointer to n^dim velocities c (double, x1 fastest, then x2, x3), c > 0.
 * omega    angular frequency omega > 0 (Sec. 1).
 * n        grid points per axis; odd, so that the two fronts meet at the middle
 *          layer (n+1)/2 (Sec. 2.3); n <= 32767 in 2D (HS_EUNSUPPORTED above).
 * dim      2, or 3 for the 7-point operator of Sec. 4 (Eq. helmd3) on n^3 points with
 *          the slab sweep of Algorithms 5 and 6 (two fronts in x3, d layers per step;
 *          each slab solved by a nested-dissection multifrontal factorisation of
 *          the (x1, x2) plane; n <= 255).
 * pml_width         b_p: boundary PML width in grid points, eta = b_p h (Eq. sigma).
 * moving_pml_width  b: moving PML width in grid points (Eq. helma), 1 <= b <= b_p + 1.
 * opt      NULL for defaults.
 * stream   stream for the setup kernels; the call synchronises it before returning
 *          (unless opt->async_setup, see there).
 * out      receives the plan.
 *
 * Every subproblem H_m (the front F, the end E, every d-layer block of both
 * fronts and the middle layer) is factored in one batched launch; windows
 * taller than 32 rows return HS_EUNSUPPORTED.  HS_EBREAKDOWN reports a zero
 * pivot.  The plan keeps a copy of c; the caller may free it after return.
 */
int hs_setup(const double* c, double omega, int n, int dim, int pml_width, int moving_pml_width,
             const hs_options* opt, void* stream, hs_plan** out);

/*
 * hs_setup_batched -- hs_setup for nprob independent problems of any sizes
 * n[k] (Algorithm 3 for each; the subproblems of all of them are independent,
 * Sec. 2.3) with shared widths and options.  c[k] is a HOST pointer to the
 * n[k]*n[k] velocities of problem k and omega[k] its frequency.  All chunk
 * factorisations of all problems run in one persistent launch, and all
 * separator systems in a second one.  On success plans[k] receives problem
 * k's plan (each later used and destroyed on its own); on any error no plan
 * is returned and nothing stays allocated.
 */
int hs_setup_batched(int nprob, const double* const* c, const double* omega, const int* n, int dim,
                     int pml_width, int moving_pml_width, const hs_options* opt, void* stream,
                     hs_plan** plans);

/*
 * hs_setup_batched_opts -- hs_setup_batched with options per problem: opts
 * points to nprob hs_options (problem k uses opts[k]), so that problems of
 * very different sizes can each reserve their own max_nrhs and chunk length
 * in the same launch.  All entries must name the same factor_prec
 * (HS_EINVAL otherwise); everything else is as for hs_setup_batched.
 */
int hs_setup_batched_opts(int nprob, const double* const* c, const double* omega, const int* n, int dim,
                          int pml_width, int moving_pml_width, const hs_options* opts, void* stream,
                          hs_plan** plans);

/*
 * hs_apply -- z = M_alpha r (Algorithm 4 with two fronts, Sec. 2.3).
 * r, z     device vectors of nrhs RHS (layout above), dtype HS_C64 or HS_C128;
 *          r and z may alias.  1 <= nrhs <= opt.max_nrhs.
 * The sweep runs in the plan's factor precision; dtype only sets the I/O type.
 */
int hs_apply(hs_plan* plan, const void* r, void* z, int nrhs, int dtype, void* stream);

/*
 * hs_apply_noalloc -- z = M_alpha r like hs_apply, for callers that must not
 * allocate device memory when they apply the preconditioner (applications
 * that hand all free device memory to their own pool at start-up,
 * latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation, hosts that forbid a library from allocating after
 * initialisation).  The paper has no counterpart; this is a deployment
 * variant of the same sweep.
 *
 * It allocates nothing: all temporaries (working vector, chunk store,
 * separator buffers) live in one file-scope device array of 32 MiB that every
 * device loading the library holds until the process exits.  The plan is
 * only read (its factors and tables); its own workspace is not touched, so
 * hs_apply, hs_solve or hs_matvec on the same plan may run at the same time
 * as this call.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Calls of this entry point share the array
 * and it keeps the last call's contents (nothing in it needs to start at
 * zero), so two hs_apply_noalloc calls that overlap on the GPU race:
 * serialise them.  Result: bit for bit that of hs_apply (same kernels, same
 * launch shapes).
 *
 * Arguments as hs_apply (2D plans; HS_EUNSUPPORTED for 3D).  Returns HS_EINVAL
 * when nrhs is outside 1..max_nrhs, when the current device is not the one
 * the plan was set up on, or when the problem does not fit:
 * n*n*nrhs + 2*n*nrhs*Wmax + 8*P*nrhs*Wmax elements of the factor precision
 * (Wmax <= 32 the padded window height, P the number of x1 chunks), each
 * rounded up to 256 bytes, must not exceed 32 MiB (for example n = 511 with
 * up to 13 right-hand sides in complex64).
 */
int hs_apply_noalloc(hs_plan* plan, const void* r, void* z, int nrhs, int dtype, void* stream);

/*
 * hs_apply_batched -- z[k] = M_alpha^(k) r[k] for nprob distinct plans, as
 * one CUDA graph whose per-problem stage chains run concurrently (small
 * problems alone cannot fill the GPU).  The graph is captured on the first
 * call for a given list of (plan, r, z, nrhs) and dtype and replayed after;
 * destroying any of the plans drops it.  r[k], z[k]: device vectors of
 * nrhs[k] RHS of plan k (1 <= nrhs[k] <= its max_nrhs), may alias.  A plan
 * may appear once only (HS_EINVAL otherwise).
 */
int hs_apply_batched(int nprob, hs_plan* const* plans, const void* const* r, void* const* z, const int* nrhs,
                     int dtype, void* stream);

/*
 * hs_autotune -- pick the tile shape of the sweep for one problem shape by
 * timing: the x1 chunk length of the subproblem solves (the chunk count sets
 * the CTAs per front of every sweep stage) and the RHS per CTA of the
 * separator solve (1, 2 or 4).  For each candidate length it sets up the
 * problem and, for each grouping, times hs_apply of nrhs RHS with CUDA events
 * on `stream`.  Writes the fastest pair to *best_chunk and *best_sep (when not
 * NULL) and its time per application in ms to *best_ms (when not NULL).
 * When opt->tune_cache is set, appends the result to that text file under the
 * key (n, pml_width, moving_pml_width, layers_per_step, factor_prec, nrhs),
 * which later hs_setup calls with chunk = 0 and max_nrhs = nrhs read.  c is a
 * HOST pointer as in hs_setup.  2D plans only (HS_EUNSUPPORTED for dim 3).
 */
int hs_autotune(const double* c, double omega, int n, int dim, int pml_width, int moving_pml_width,
                const hs_options* opt, int nrhs, void* stream, int* best_chunk, double* best_ms, int* best_sep);

/*
 * hs_matvec -- y = A x with the Eq. helmd operator (alpha = 0).
 * dtype HS_C128 computes in FP64, HS_C64 in FP32.  x and y must not alias.
 */
int hs_matvec(hs_plan* plan, const void* x, void* y, int nrhs, int dtype, void* stream);

/*
 * hs_solve -- solve A u = f for nrhs RHS with right-preconditioned flexible
 * GMRES(m) (Sec. 2.3 uses GMRES on M_alpha A; the flexible right form lets the
 * true residual decide): FP64-class true residual and iterate (double-float
 * for complex64 2D plans, FP64 otherwise), Arnoldi basis per
 * opt.krylov_basis, preconditioner in the plan's factor precision.  The RHS advance in lock
 * step; each stops when ||f - A u|| <= tol ||f|| (FP64, recomputed at every
 * restart and at the end).
 * f, u     device HS_C128 vectors; u is the initial guess on entry and the
 *          solution on return.
 * tol      relative residual tolerance (> 0).  maxit: max Arnoldi steps.
 * info     optional host struct (may be NULL).
 * Synchronises `stream`.  Returns HS_ENOCONV if some RHS did not converge.
 */
int hs_solve(hs_plan* plan, const void* f, void* u, int nrhs, double tol, int maxit,
             hs_solve_info* info, void* stream);

/*
 * Convolutional post-correction of the sweep (no counterpart in the paper; a
 * learned addition used inside flexible GMRES, judged by the FP64 residual).
 * For a sweep output x = M_alpha r:
 *
 *   z <- z + s N(x / s),   s = sqrt(mean over points of |x|^2) per RHS,
 *   N = conv3x3(2->32) + b1, ReLU, conv3x3(32->32) + b2, ReLU, conv3x3(32->2) + b3,
 *
 * on the n x n grid of each RHS (rows x2, columns x1, zero padding), input
 * channels (Re, Im) of x/s, output channels (Re, Im) of the correction; it
 * is trained on the sweep's error e = A^{-1} r - M_alpha r.
 * Parameters: HS_CNN_NPARAM floats in the order W1[3][3][2][32], b1[32],
 * W2[3][3][32][32], b2[32], W3[3][3][32][2], b3[2]; W[ky][kx][ci][co]
 * multiplies input channel ci at row offset ky-1 and column offset kx-1.
 * Activations are stored in bfloat16, weights used as their bfloat16
 * roundings of FP32 masters; arithmetic in FP32.
 */
#define HS_CNN_NPARAM 10434
typedef struct hs_cnn hs_cnn;

/* Create a network from HOST parameters (copied).  */
int hs_cnn_create(const float* params, hs_cnn** out);
/* Copy the current FP32 parameters to HOST memory (HS_CNN_NPARAM floats). */
int hs_cnn_get_params(const hs_cnn* net, float* params);
/* 1: layer 2 on the tensor cores (tcgen05); 0: FP32 reference kernel. */
int hs_cnn_set_mode(hs_cnn* net, int tensor_cores);
/* z += s N(x / s) for nrhs device vectors of n x n points (ABI layout, dtype
 * HS_C64 or HS_C128); x and z may alias (the usual use: z = x = M_alpha r).
 * Workspace (two bf16 activation tensors of nrhs*n*n*32 values) is
 * allocated on first use and kept. */
int hs_cnn_apply(hs_cnn* net, const void* x, void* z, int nrhs, int n, int dtype, void* stream);
/* Loss L = mean over points and RHS of |N(x/s) - e/s|^2 for training pairs
 * (x, e) = (M_alpha r, A^{-1} r - M_alpha r) (device, ABI layout) and its
 * gradient dL/dtheta (HOST, may be NULL).  Synchronises the stream. */
int hs_cnn_gradient(hs_cnn* net, const void* x, const void* e, int nrhs, int n, int dtype, double* loss,
                    float* grad, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * gradient of the same loss; *loss (if not NULL) gets the loss before the
 * step (synchronises the stream). */
int hs_cnn_train_step(hs_cnn* net, const void* x, const void* e, int nrhs, int n, int dtype, double lr,
                      double* loss, void* stream);
/* One Adam step on the residual loss L = mean over RHS of |A c - rho|^2 / |rho|^2,
 * c = s N(x/s), for sweep outputs x = M_alpha v and their residuals
 * rho = v - A x (complex64 device vectors of plan's n x n grid, ABI layout;
 * A is the plan's Eq. helmd operator): the quantity the solver's judge
 * compares.  *loss (if not NULL) gets L before the step (synchronises). */
int hs_cnn_train_step_residual(hs_cnn* net, hs_plan* plan, const void* x, const void* rho, int nrhs, double lr,
                               double* loss, void* stream);
/* Wait for `stream` and report a device error recorded by the network's
 * tensor-core kernel (HS_ETIMEOUT after an expired bounded wait). */
int hs_cnn_sync(hs_cnn* net, void* stream);
int hs_cnn_destroy(hs_cnn* net);
/* Let hs_solve post-correct its preconditioner with the network (NULL
 * detaches).  For each Arnoldi direction v and RHS the solver forms the
 * sweep output x = M_alpha v and the correction c = s N(x / s), and the FP64
 * residual decides: z = x + c is kept where |v - A (x + c)| < |v - A x|, else
 * the plain sweep output z = x (one extra matvec per direction).  The network
 * must outlive its use. */
int hs_attach_cnn(hs_plan* plan, hs_cnn* net);

/* Wait for the plan's work on `stream` and report any recorded device error. */
int hs_sync(hs_plan* plan, void* stream);

/* Status recorded by device kernels since setup (HS_OK if none). */
int hs_last_device_status(hs_plan* plan);

/* Arithmetic of a 3D plan's setup (Sec. 4.2, Algorithm 5), for rooflines:
 * real flops of the frontal Schur-update GEMMs (L = F21 G, F22 -= L F12;
 * 8 per complex multiply-add) and of the front pivot-block inversions
 * (8 S^3 for an S x S block).  HOST outputs (either may be NULL); 0 for 2D
 * plans. */
int hs_setup_flops(const hs_plan* plan, double* gemm_flops, double* inverse_flops);

/* Bytes of device memory owned by the plan (factors, tables, sweep workspace). */
long long hs_plan_bytes(const hs_plan* plan);

/*
 * hs_solve draws its Krylov basis (restart+1 FP64 vectors and restart
 * preconditioned vectors of nrhs RHS) from one device buffer shared by the
 * whole process; it grows on demand and is kept between calls so that
 * repeated solves do not reallocate.  Solves from several host threads take
 * turns on it.  hs_release_workspace() frees it (no solve may be running),
 * and also returns to the device the memory that destroyed 2D plans left in
 * the library's plan pool (plan buffers come from a stream-ordered pool that
 * keeps freed memory, so that setting up a new plan after destroying one does
 * not map its memory again).
 */
int hs_release_workspace(void);

/* Diagnostic: number of kernels libhs has launched in this process. */
long long hs_kernel_launches(void);

/* Free the plan and all device memory it owns (on the plan's device, whichever
 * device is current; 2D plan buffers return to the library's plan pool, from
 * which the next plan draws them, until hs_release_workspace()).  NULL is
 * accepted. */
int hs_destroy(hs_plan* plan);

/* Static description of a status code. */
const char* hs_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* HS_H_ */
