/*
 * aao.h -- C ABI of the GB300 all-at-once alpha-circulant solver (libaao.so).
 *
 * Problem (Eq. 1 of Tabeart, Gurol, Pearson, Weaver, "Block alpha-circulant
 * preconditioners for all-at-once diffusion-based covariance operators"):
 *
 *     script-A x = b,   script-A = block lower bidiagonal with A on the
 *     diagonal and -I_N below it;  (script-A x)_t = A x_t - x_{t-1}, x_0 = 0.
 *
 * A = I + K is the SPD Neumann finite-volume diffusion matrix on a 1D/2D/3D
 * cell grid: (K v)_c = sum over the faces f of cell c of kappa_f (v_c - v_nbr).
 * There are no boundary faces, so the constant vector is in ker K and the
 * smallest eigenvalue of A is mu_min = 1.
 *
 * Preconditioner: P_alpha (Eq. 2) applied through Eq. 5 -- alpha-scaling,
 * length-ell DFT over the time blocks, ell shifted solves
 * (A - lambda_j I) y_j = v_j (Eq. 7) each approximated by a fixed number p of
 * Chebyshev semi-iteration steps over the segment of Lemma 2 (P_NC1,
 * Section 5), inverse DFT and unscaling.  Only the ell/2+1 frequencies that
 * are distinct for real input and even ell are computed (Section 3).
 * Outer solver: right-preconditioned flexible GMRES with modified
 * Gram-Schmidt (classical, once or twice, on request); convergence is the paper's
 * relative residual ||b - script-A x|| / ||b|| (Section 5), certified by an
 * explicit FP64 residual.
 *
 * Layout of every block vector (b, x, r, z, y): "block-major" as in Eq. 1,
 * ell blocks of N doubles, block t-1 at offset (t-1)*N; within a block cells
 * are ordered x fastest: c = i + n0*(j + n1*k).
 *
 * Memory: pointers may be device pointers or host pointers (pageable or
 * pinned); the library detects which (cudaPointerGetAttributes) and stages
 * host data through buffers it owns, with the copies on the handle's stream.
 * The caller owns every pointer it passes and keeps device buffers alive
 * until the call returns (all calls synchronise the handle's stream before
 * returning, except where noted).  The library owns all workspace.  Block
 * vectors must be 8-byte aligned (AAO_EINVAL otherwise); an output written
 * two doubles at a time (z of aao_precond_apply) that is device memory but
 * not 16-byte aligned is staged like host memory and copied on the device.
 *
 * Threads and streams: one handle is used by one host thread at a time; all
 * device work of a handle is ordered on the stream given at creation.
 *
 * Errors: every int-returning call returns an AAO_* status.  On failure a
 * one-line message is available from aao_last_error(h) (or
 * aao_last_create_error() when aao_create itself failed).  There is no CPU
 * fallback: without a usable CUDA device every call fails with AAO_ECUDA.
 */
#ifndef AAO_H
#define AAO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define AAO_OK 0        /* success                                              */
#define AAO_EINVAL 1    /* invalid argument (sizes, ell, alpha, kappa, pointers) */
#define AAO_ENOMEM 2    /* device or host allocation failed                     */
#define AAO_ECUDA 3     /* a CUDA call failed (no device, launch error, ...)    */
#define AAO_ENOTCONV 4  /* solve hit max_outer; x holds the last iterate        */
#define AAO_ENUMERIC 5  /* a NaN or Inf appeared in a residual or norm          */
#define AAO_ETIMEOUT 6  /* a bounded device-side wait expired (see aao_set_wait_limit) */

/* ---- precision modes ----------------------------------------------------- */
#define AAO_FP64 0      /* every step in FP64                                   */
#define AAO_MIXED 1     /* DFT, Chebyshev sweeps, inverse DFT in (complex) FP32;
                           script-A, Arnoldi, Givens, residuals in FP64         */

/* ---- limits -------------------------------------------------------------- */
#define AAO_ORTH_CGS 0   /* classical Gram-Schmidt, one pass                      */
#define AAO_ORTH_CGS2 1  /* classical Gram-Schmidt with one re-orthogonalisation  */
#define AAO_ORTH_MGS 2   /* modified Gram-Schmidt (one fused kernel per vector)   */
#define AAO_MAX_ELL 16      /* ell must be even, 4 <= ell <= AAO_MAX_ELL        */
#define AAO_MAX_RESTART 64  /* Krylov cycle length limit                        */
#define AAO_MAX_HIST 512    /* residual history entries kept in aao_stats       */

typedef struct aao_ctx* aao_handle;
typedef struct aao_batch_ctx* aao_batch;

/* Options for aao_create.  Fill with aao_default_options first. */
typedef struct {
  int32_t prec;            /* AAO_FP64 or AAO_MIXED (default AAO_MIXED)                 */
  int32_t inner_its;       /* p >= 1: Chebyshev steps per frequency (default 20)         */
  int32_t restart;         /* Krylov cycle length m, 1..AAO_MAX_RESTART (default 64)     */
  int32_t orth;            /* Arnoldi orthogonalisation: AAO_ORTH_MGS (default),
                              AAO_ORTH_CGS2 or AAO_ORTH_CGS                           */
  double mu_max_override;  /* > 0: upper spectral bound of A to use instead of the
                              Gershgorin bound max_c (1 + 2 sum_f kappa_f) (default 0)   */
  void* stream;            /* cudaStream_t for all work of the handle (NULL = default)  */
} aao_options;

/* Statistics of the last aao_solve (Section 5 counts A-matvecs per outer
 * iteration: ell for script-A, ell*p for the preconditioner, Table 1). */
typedef struct {
  int32_t outer_its;       /* Arnoldi steps taken (all cycles)                          */
  int32_t cycles;          /* Krylov cycles (restarts + 1)                              */
  int32_t converged;       /* 1 if the explicit residual met tol                        */
  int32_t n_hist;          /* entries in hist                                           */
  int64_t a_matvecs;       /* real A-matvec equivalents, counted as in Table 1         */
  double resid_est;        /* last Givens estimate of ||b - script-A x|| / ||b||        */
  double resid_explicit;   /* explicit FP64 ||b - script-A x|| / ||b|| at return        */
  double mu_min;           /* lower spectral bound of A used (1 for Neumann)            */
  double mu_max;           /* upper spectral bound of A used                            */
  double hist[AAO_MAX_HIST]; /* relative residual estimate after each Arnoldi step      */
} aao_stats;

/* Kernel classes timed by the built-in profiler (aao_profile_*). */
#define AAO_PROF_DFT 0        /* forward transform (Eq. 5's U* Gamma)                      */
#define AAO_PROF_STEP_FIRST 1 /* Chebyshev step k = 1 (x_1 = bhat/theta); on the 2D mixed
                                 path one launch with the forward transform               */
#define AAO_PROF_STEP_SECOND 2 /* Chebyshev step k = 2                                     */
#define AAO_PROF_STEP_MID 3   /* single Chebyshev steps 3 <= k <= p-1 (k = p-1 when it
                                 writes x_p for a separate inverse transform)             */
#define AAO_PROF_STEP_LAST 4  /* the inverse transform of x_p (mixed precision with an
                                 even cell count), else the last Chebyshev step fused with
                                 the inverse transform                                    */
#define AAO_PROF_MATVEC 5     /* script-A matvec and explicit residual                      */
#define AAO_PROF_ORTH 6       /* Gram-Schmidt multi-dots, updates and their reductions     */
#define AAO_PROF_STEP_PAIR 7  /* two fused Chebyshev steps (2D mixed path)                 */
#define AAO_PROF_STEP_QUAD 8  /* four fused Chebyshev steps (2D mixed path)                */
#define AAO_NPROF 9

/* Accumulated device time of each kernel class, from CUDA events recorded on
 * the handle's stream around every launch while profiling is on (around the
 * warp-strip launches of one apply together, which run back to back), with
 * the algorithmic bytes each launch must move (reads + writes of its operands,
 * every value once). */
typedef struct {
  int64_t launches[AAO_NPROF];
  double ms[AAO_NPROF];
  double bytes[AAO_NPROF];
} aao_profile;

/* Fill *opt with the defaults listed above.  Never fails. */
void aao_default_options(aao_options* opt);

/*
 * Create a solver for one instance (Eq. 1 with Eq. 2's preconditioner).
 *   h      out: new handle (NULL on failure).
 *   dim    1, 2 or 3.
 *   n      cells per axis n[0] (x), n[1] (y), n[2] (z); unused axes must be 1;
 *          N = n0*n1*n2 >= 1.
 *   kx     interior x-face diffusivities, (n2, n1, n0-1) x fastest, doubles;
 *   ky     y-faces (n2, n1-1, n0); kz z-faces (n2-1, n1, n0).  A pointer for
 *          an axis with no faces may be NULL.  Host or device memory; copied.
 *          Every value must be finite and > 0.
 *   ell    number of time blocks: even, 4 <= ell <= AAO_MAX_ELL (Section 1
 *          takes ell > 2 even; conjugate symmetry needs ell even, Section 3).
 *   alpha  0 < alpha < mu_min^ell = 1 (Corollary 1 and Lemma 1 need
 *          alpha != mu_j^ell; alpha = 1 makes P_alpha singular here).
 *   opt    options or NULL for the defaults.
 * Sets up: Gershgorin mu_max (or the override), shifts lambda_j, scalings,
 * Chebyshev coefficient tables (host FP64, uploaded as FP32 and/or FP64),
 * and the workspace (about (2m+3) ell N doubles plus 3 ell N Chebyshev
 * values).  Returns AAO_EINVAL, AAO_ENOMEM or AAO_ECUDA on failure.
 */
int aao_create(aao_handle* h, int dim, const int64_t n[3], const double* kx,
               const double* ky, const double* kz, int ell, double alpha,
               const aao_options* opt);

/* y = script-A x (Eq. 1), FP64.  x, y: ell*N doubles, block-major, distinct. */
int aao_matvec(aao_handle h, const double* x, double* y);

/* z = P_NC^{-1} r: Eq. 5 with p Chebyshev steps per frequency (NC1), in the
 * handle's precision.  r, z: ell*N doubles, block-major, distinct. */
int aao_precond_apply(aao_handle h, const double* r, double* z);

/*
 * Solve script-A x = b by right-preconditioned FGMRES(m) with P_NC.
 *   b          ell*N doubles (the paper's b has only b_1 non-zero; any b works).
 *   x          in: initial guess if use_x0 != 0, else ignored (x_0 = 0,
 *              Section 5); out: the solution iterate.
 *   tol        target for the explicit relative residual ||b - script-A x||/||b||.
 *   max_outer  limit on Arnoldi steps over all cycles (>= 1).
 *   inner_its  p for this solve (> 0), or 0 to keep the handle's value.
 * Returns AAO_OK when the explicit residual is below tol, AAO_ENOTCONV when
 * max_outer was reached first (x then holds the last iterate), AAO_ENUMERIC
 * on NaN/Inf.  Statistics: aao_get_stats.
 */
int aao_solve(aao_handle h, const double* b, double* x, double tol, int max_outer,
              int inner_its, int use_x0);

/* Run exactly k Arnoldi steps in one cycle from x_0 = 0 and form x (no early
 * stop); used to compare iterates step by step with a reference.  Same
 * arguments as aao_solve.  Returns AAO_OK (or an error). */
int aao_solve_fixed(aao_handle h, const double* b, double* x, int k, int inner_its);

/*
 * Per-frequency inner budgets (P_NC2, Section 5 and Algorithm 1): frequency j
 * (shift lambda_{j+1}) runs p[j] Chebyshev steps instead of the handle's
 * common count.  p has ell entries with p[j] == p[ell-j] (conjugate shifts
 * share a budget, Section 3); p[j] = 0 gives y_j = 0.  Frequencies whose
 * budget is spent keep their iterate while the others continue (their
 * recurrence coefficients are set to zero), so an apply runs max_j p[j]
 * steps.  Stays in force until aao_solve is called with inner_its > 0.
 */
int aao_set_inner_alloc(aao_handle h, const int32_t* p, int ell);

/*
 * Kernel that runs the fused four-step Chebyshev sweeps of the 2D mixed path
 * (no counterpart in the paper; both compute the same steps of Eq. 7):
 *   AAO_STEP_AUTO  the kernel and configuration chosen by the autotuner or the
 *                  tune cache (aao_autotune, aao_set_tune_cache), else the
 *                  warp-strip kernel with its default configuration;
 *   AAO_STEP_TILE  the shared-memory tile kernel (one CTA per 120 x 16 tile);
 *   AAO_STEP_TMA   the persistent TMA-fed kernel (one CTA per SM);
 *   AAO_STEP_STREAM the warp-strip kernel streamed along y: S steps per launch
 *                  (aao_set_stream_config), one warp per 64-column strip of an
 *                  H-row segment, inputs prefetched by per-lane cp.async rings.
 * Returns AAO_EINVAL for an unknown kind, or when the handle has no fused
 * 2D path (FP64, 1D/3D, n0 % 4 != 0) or, for AAO_STEP_TMA, no descriptors.
 * A TMA wait in the persistent kernel that does not finish within the wait
 * limit (about a second of SM clock by default) makes the enclosing
 * aao_solve / aao_solve_ci / aao_precond_apply return AAO_ETIMEOUT; the
 * kernel first lets its own copies land, so the handle stays usable.  The
 * fault flag is per handle.
 */
#define AAO_STEP_AUTO 0
#define AAO_STEP_TILE 1
#define AAO_STEP_TMA 2
#define AAO_STEP_STREAM 3
int aao_set_step_kernel(aao_handle h, int kind);
/*
 * Configuration of the warp-strip kernel (AAO_STEP_STREAM): S fused Chebyshev
 * steps per launch (the halo width; 2 or 4), H interior rows per segment
 * (1 <= H <= 4096), D rows prefetched ahead (3 or 4; 5 with S = 4 and NW = 8) and
 * NW warps per CTA.
 * H + 2S a multiple of 6: the S levels of a row step advance in lockstep (S = 4:
 * NW 6, 8 or 12; S = 2: NW 8, 12 or 16).  S = 4 and H + 9 a multiple of 6: the
 * skewed schedule, where levels 3 and 4 trail level 2 by one more row so that a
 * row step holds two independent chains of levels (NW 8; one more row step per
 * segment; the same arithmetic, bit for bit).  The default without a tune cache
 * is S = 4 on the skewed schedule, D = 5, NW = 8 and the segment height that
 * fills one round of the device's warps.  No counterpart in the paper: these
 * are launch parameters of this library's kernel (Eq. 7's steps are
 * unchanged).  AAO_EINVAL for an unsupported combination.
 * aao_get_stream_config writes (S, H, D, NW) to out[0..3].
 *
 * With the warp-strip kernel the sweep runs steps 2 .. p-1 (step 1 and, when
 * their count p - 2 is odd, step 2 run alone): launches of S steps, and with
 * S = 4 and a remainder of two steps one two-step launch configured by
 * aao_set_stream_tail (H + 4 a multiple of 6, D in {3, 4}, NW in {8, 12, 16};
 * default: D = 3, NW = 16 and the height that fills one round of the device's
 * warps).  The final launch writes x_p alone and a separate kernel applies
 * Eq. 5's inverse transform and Gamma^{-1} to it.  aao_get_stream_tail writes
 * (H, D, NW) to out[0..2].
 */
int aao_set_stream_config(aao_handle h, int S, int H, int D, int NW);
int aao_get_stream_config(aao_handle h, int32_t out[4]);
int aao_set_stream_tail(aao_handle h, int H, int D, int NW);
int aao_get_stream_tail(aao_handle h, int32_t out[3]);

/*
 * Autotuner of the fused sweep (no counterpart in the paper: the method's steps are
 * unchanged; only which kernel runs them, and with which launch parameters, is chosen).
 * Candidates: AAO_STEP_TILE, AAO_STEP_TMA, and AAO_STEP_STREAM with halo depth S in {2, 4},
 * segment heights that fill one to three rounds of the device's warps (and one segment per
 * strip), each supported D (3 to 5) and NW.  Each candidate runs reps + 1 preconditioner
 * applies on the handle's own staging buffers (the first untimed) and is timed by CUDA events
 * on the handle's stream; the fastest becomes what AAO_STEP_AUTO selects on h.  When the
 * winner is the warp-strip kernel with S = 4 and the sweep ends in a two-step launch, the
 * two-step configurations (NW in {8, 12, 16}, D in {3, 4}, one to three rounds of units) are
 * timed next under the winner (entries with tail = 1) and the fastest becomes h's tail
 * (aao_set_stream_tail).
 *   results, max_results: optional array receiving up to max_results candidates with their
 *                  mean time per apply in microseconds (us_per_apply < 0: did not run);
 *   n_results:     optional, receives the number of candidates; best: optional, the winner.
 * The handle needs the fused 2D mixed path (n0 % 4 == 0), P_NC and inner_its >= 3, else
 * AAO_EINVAL.  Synchronises the handle's stream; allocates the staging buffers if absent.
 */
typedef struct {
  int32_t kind;         /* AAO_STEP_TILE, AAO_STEP_TMA or AAO_STEP_STREAM */
  int32_t S, H, D, NW;  /* warp-strip configuration (S = 4 and zeros for the other kernels) */
  int32_t tail;         /* 1: a two-step final launch (S = 2) timed under the best sweep */
  double us_per_apply;  /* mean time of one preconditioner apply */
} aao_tune_entry;
int aao_autotune(aao_handle h, int reps, aao_tune_entry* results, int max_results, int* n_results,
                 aao_tune_entry* best);
/*
 * Tune cache: a JSON file {"version": 1, "entries": [{"device", "dim", "n": [n0, n1, n2],
 * "ell", "prec": "mixed" | "fp64", "p", "kernel": "tile" | "tma" | "stream", "S", "H", "D",
 * "NW", ...}]} (written by the package's tune module).  aao_set_tune_cache sets its path for
 * every later aao_create in the process (NULL: none; without a call, the environment
 * variable AAO_TUNE_CACHE is used); aao_create applies the entry matching the device name,
 * dim, n, ell and precision (one with the same inner_its preferred) to AAO_STEP_AUTO, and
 * without one uses the default of aao_set_stream_config (S = 4 on the skewed schedule,
 * D = 5, NW = 8, the segment height that fills one round of the device's warps).
 * aao_tune_lookup performs that lookup on the host alone (no device needed): returns 1 and
 * fills out = (kind, S, H, D, NW) when an entry matches, 0 when none does, and -AAO_EINVAL
 * when the file cannot be read or parsed.  device NULL matches any device.
 * aao_get_tuning writes (kernel in use, S, H, D, NW, 1 if chosen by the tuner or the cache).
 */
int aao_set_tune_cache(const char* path);
int aao_tune_lookup(const char* path, const char* device, int dim, const int64_t n[3], int ell, int prec, int p,
                    int32_t out[5]);
int aao_get_tuning(aao_handle h, int32_t out[6]);
/*
 * Preconditioner of the outer solve (aao_solve, aao_solve_ci, aao_precond_apply):
 *   AAO_PRECOND_NC         P_NC, Eq. 5 with Chebyshev inner solves (default);
 *   AAO_PRECOND_EXACT_DCT  the paper's best-case P_alpha applied exactly (Section 5's
 *                          comparison), through A = X Phi X^T (Section 2.2): for face
 *                          diffusivities that are constant along each axis, X is the
 *                          orthonormal DCT-II along every axis and
 *                          Phi = 1 + sum_a kappa_a 4 sin^2(pi k_a / (2 n_a)).  The spatial
 *                          transforms are this library's kernels (a fast DCT through one FFT
 *                          per line for power-of-two axes, direct sums otherwise); FP64
 *                          handles only.
 *   AAO_PRECOND_SP         P_SP (Section 4): the real shifts (frequencies 0 and ell/2) by
 *                          p steps of CG on A - lambda I, each complex shift by p steps of
 *                          MINRES on the saddle-point system of twice the size with the
 *                          block-diagonal preconditioner P_D (Section 4's theorem); the SPD
 *                          blocks are applied by one V-cycle of this library's aggregation
 *                          multigrid (the paper uses an algebraic multigrid, HSL_MI20):
 *                          2 x 2 (3D: 2 x 2 x 2) aggregates, Galerkin coarse levels.
 *                          p = the handle's inner_its.  FP64 handles, 1D, 2D and 3D grids.
 * Returns AAO_EINVAL for an unknown mode, a mixed-precision handle (P_SP and the exact mode)
 * or face diffusivities that vary along an axis (exact mode, relative spread > 1e-12).  With the
 * exact mode the statistics count ell A-products per outer iteration (P_alpha^{-1} uses none);
 * with P_SP, ell + ell p (CG: one product per step on two real shifts; MINRES: two per step on
 * the ell/2 - 1 complex shifts that conjugate symmetry leaves).
 */
#define AAO_PRECOND_NC 0
#define AAO_PRECOND_EXACT_DCT 1
#define AAO_PRECOND_SP 2
int aao_set_precond_mode(aao_handle h, int mode);

/*
 * Bound, in SM clock cycles, of each wait of the persistent TMA kernel on its
 * copies (no counterpart in the paper).  Default 2e9 (about a second).  A
 * small value makes the waits expire before the copies land: the kernel then
 * records the expiry, waits for its copies with the default bound, returns,
 * and the call reports AAO_ETIMEOUT.  This is the fault-injection hook for
 * testing that path without faulting or hanging the GPU.  Returns AAO_EINVAL
 * for cycles < 0.
 */
int aao_set_wait_limit(aao_handle h, int64_t cycles);

/* The kernel in use: AAO_STEP_TMA or AAO_STEP_TILE on the fused 2D path,
 * AAO_STEP_AUTO when the handle has none; -1 for a NULL handle. */
int aao_get_step_kernel(aao_handle h);

/*
 * Algorithm 1 of the paper, on the host: share ell * nx * eta inner
 * iterations among the ell shifted problems in proportion to
 * ln(sigma_1) / ln(sigma_j), sigma_j from Theorem 4 on [mu_min, mu_max], and
 * round each share down.  out receives ell counts.  Returns AAO_EINVAL on bad
 * arguments (ell odd, mu_max <= mu_min, alpha^(1/ell) >= mu_min, ...).
 */
int aao_assign_iterations(int ell, int64_t nx, double mu_max, double mu_min, double alpha, double eta,
                          int32_t* out);

/*
 * The paper's own outer solver: Chebyshev semi-iteration on the
 * preconditioned system P^{-1} script-A x = P^{-1} b (Eq. 3, Section 5) over
 * the eigenvalue interval [l_min, l_max] of P^{-1} script-A.  Passing
 * l_min = l_max = 0 takes Corollary 1's interval
 * [1, mu_N^ell / (mu_N^ell - alpha)] for the exact P_alpha, kept unchanged for
 * the inexact P_NC as in Section 5.  Each iteration costs one script-A product
 * and one preconditioner apply (Table 1).  The residual is updated as
 * r <- r - script-A d in FP64; convergence is ||b - script-A x|| / ||b|| < tol,
 * certified by an explicit residual at the end.
 *   fixed_its > 0 runs exactly that many iterations (tol ignored).
 * Other arguments as aao_solve.  Needs restart >= 2 (it uses the Krylov
 * workspace).  Returns AAO_ENOTCONV if max_outer iterations do not reach tol
 * (CI can stagnate when P_NC is far from P_alpha).
 */
int aao_solve_ci(aao_handle h, const double* b, double* x, double tol, int max_outer, int inner_its, int use_x0,
                 double l_min, double l_max, int fixed_its);

/*
 * Batched solve: many independent instances of Eq. 1 (different grids, ell,
 * alpha, diffusivities and right-hand sides) solved together.  All members
 * advance in lockstep through right-preconditioned FGMRES; every phase of an
 * Arnoldi step (transform, the Chebyshev steps, matvec, each modified
 * Gram-Schmidt step, Givens) is one launch over all members.  The fused
 * Chebyshev sweeps (four steps per launch while they fit before the last one)
 * are one persistent warp-strip launch over the units (member, frequency
 * pair, segment, strip) of every member whatever its ell, which the warps take
 * from a device work queue; the transforms and single steps run one launch per
 * distinct ell, each block mapped to an (instance, tile) pair.  Members that
 * have converged skip their work.  With use_graphs != 0 each Arnoldi step is
 * captured once as a CUDA graph and replayed.  The paper solves one instance
 * at a time; batching is this library's addition for covariance operators
 * applied to many fields at once.
 *   members    count handles created with AAO_MIXED, all 2D or all 3D (3D:
 *              inner_its >= 3), n[0] % 4 == 0, and the same inner_its (>= 2)
 *              and restart; they must outlive the
 *              batch, and the batch uses their workspace (do not use the
 *              members concurrently with a batched solve).  The batch
 *              orthogonalises by modified Gram-Schmidt when every member
 *              uses AAO_ORTH_MGS (the default), else by CGS2.
 * The batch has its own non-blocking stream.
 */
int aao_batch_create(aao_batch* hb, int count, const aao_handle* members, int use_graphs);

/*
 * Solve every member i: script-A_i x[i] = b[i] from x_0 = 0 to explicit
 * relative residual < tol, at most max_outer Arnoldi steps each.  b and x
 * are arrays of count DEVICE pointers (ell_i * N_i doubles each, block-major).
 * Synchronises the device at entry and the batch stream at exit.  Returns
 * AAO_ENOTCONV if any member did not converge (all x[i] hold their iterates).
 */
int aao_batch_solve(aao_batch hb, const double* const* b, double* const* x, double tol, int max_outer);

/* Statistics of member i in the last batched solve. */
int aao_batch_get_stats(aao_batch hb, int i, aao_stats* s);

/* Message of the last failed batch call ("" if none). */
const char* aao_batch_last_error(aao_batch hb);

/* Release the batch (not its members).  NULL is allowed. */
void aao_batch_destroy(aao_batch hb);

/*
 * Fused sweep of the batch (no counterpart in the paper: launch parameters of
 * the same steps; 2D batches):
 *   AAO_STEP_STREAM  S = 4, segment height H (H + 8 a multiple of 6: the
 *                    lockstep schedule; the skewed one is the single solver's
 *                    only), D in {3, 4} and NW = 8 (the default: H = 64, D = 3, used when
 *                    inner_its >= 7).  As in the single solver: the transform
 *                    and step 1 in one launch per ell, steps 2 .. p-1 as
 *                    warp-strip launches over every member's units (step 2
 *                    alone when their count is odd; a two-step final launch,
 *                    H - 2, for a remainder of two), the final launch writing
 *                    x_p, then the inverse transform per ell;
 *   AAO_STEP_TILE    the shared-memory tile kernel, one launch per distinct
 *                    ell, single steps through step p-1 and the inverse
 *                    transform per ell (S, H, D, NW ignored; the default when
 *                    inner_its < 7);
 *   AAO_STEP_AUTO    single steps through step p-1 and the inverse transform
 *                    (every 3D batch runs these).
 * Drops the captured graphs.
 */
int aao_batch_set_sweep(aao_batch hb, int kind, int S, int H, int D, int NW);
/*
 * Event timing of the batch's Chebyshev sweeps (graphs are not used while it
 * is on; turning it on or off clears the totals).  With a fused sweep the
 * fused launches of each Arnoldi step, which run back to back, are timed as one
 * span: x_k, x_{k-1} or none, bhat and two face arrays read and two fields
 * written per launch (one, x_p, by the final launch).  With single steps
 * (every 3D batch) the steps k = 2 .. p-1 of each ell group are timed as one span of
 * p - 2 launches: x_k, x_{k-1} (none at k = 2) and bhat read and x_{k+1}
 * written per member, and the dim face arrays once per member, or once for
 * the whole group when the members share one operator.  4-byte values, over
 * the members active in each launch.  aao_batch_get_profile synchronises the
 * batch stream and writes the number of timed launches, their total
 * milliseconds and their algorithmic bytes.
 */
int aao_batch_profile_enable(aao_batch hb, int on);
int aao_batch_get_profile(aao_batch hb, int64_t* launches, double* ms, double* bytes);

/* Copy the statistics of the last solve into *s. */
int aao_get_stats(aao_handle h, aao_stats* s);

/*
 * Several right-hand sides of h's operator (Eq. 1 with the same A, ell and
 * alpha), solved together: b and x are arrays of nrhs DEVICE pointers (ell N
 * doubles each, block-major), x from x_0 = 0 to explicit relative residual <
 * tol, at most max_outer Arnoldi steps each.  The right-hand sides advance in
 * lockstep through right-preconditioned FGMRES, as a batch (aao_batch_*) of
 * views of h: each view has its own Chebyshev fields and Krylov spaces
 * (restart as h) and uses h's face coefficients, shifts and step tables, so
 * each single-step Chebyshev launch loads a tile's stencil once and applies it
 * to every active right-hand side (on 2D grids the fused sweeps are the
 * batch's warp-strip launches).  The paper solves one right-hand side at a
 * time; this is the library's form for covariance operators applied to many
 * fields.  Needs the mixed path on a 2D or 3D grid with n0 % 4 == 0, P_NC,
 * inner_its >= 3 (one count for all frequencies) and restart >= 2.  The views
 * (nrhs x (2 restart + 1) Krylov vectors) are allocated on the first call and
 * kept on h until nrhs, inner_its or the tables change, or h is destroyed.
 * Returns AAO_ENOTCONV if some right-hand side did not converge (all x[i] hold
 * their iterates); aao_multi_get_stats gives right-hand side i's statistics.
 */
int aao_solve_multi(aao_handle h, int nrhs, const double* const* b, double* const* x, double tol, int max_outer);
int aao_multi_get_stats(aao_handle h, int i, aao_stats* s);
/*
 * Event timing of the Chebyshev sweeps of aao_solve_multi on h (the batch
 * profile above, applied to the right-hand sides' batch; the totals restart
 * when the views are rebuilt).  aao_multi_get_profile writes zeros before the
 * first aao_solve_multi.
 */
int aao_multi_profile_enable(aao_handle h, int on);
int aao_multi_get_profile(aao_handle h, int64_t* launches, double* ms, double* bytes);

/* Spectral bounds used for A: mu_min and mu_max (Lemma 2's segment ends). */
int aao_get_bounds(aao_handle h, double* mu_min, double* mu_max);

/* Message of the last failed call on h ("" if none).  Valid until the next
 * call on h.  Never NULL. */
const char* aao_last_error(aao_handle h);

/* Message of the last failed aao_create in this process. */
const char* aao_last_create_error(void);

/* Turn event timing of the kernel classes on (1) or off (0) for h; either
 * way the accumulated profile is cleared.  Timing adds two event records per
 * timed launch on the handle's stream. */
int aao_profile_enable(aao_handle h, int on);

/* Synchronise h's stream, resolve the recorded events and copy the
 * accumulated profile into *out. */
int aao_profile_get(aao_handle h, aao_profile* out);

/* Number of kernels this library has launched in this process (all handles);
 * used to count device work inside a timed region. */
int64_t aao_kernel_launch_count(void);

/*
 * Preconditioner apply that allocates no device memory and needs no handle.
 * The paper has no counterpart: this exists for callers that cannot let a
 * library call cudaMalloc -- applications whose device memory is owned by
 * their own pool or held to a fixed budget on a shared GPU, and latency-bound
 * callers that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree may cause.  (aao_create allocates, so such callers cannot hold a
 * handle.)
 *
 * Computes the same z = P_NC^{-1} r as aao_precond_apply on a handle created
 * with the same arguments: the same method steps, one Chebyshev step per
 * launch.  (On 2D mixed-precision grids a handle fuses several steps per
 * launch, so the two agree to rounding, not bit for bit.)  Every temporary
 * (face coefficients, three Chebyshev field buffers, reduction partials)
 * lives in one fixed 16 MiB array in the library's device memory, which every
 * GPU that loads the library holds until the process exits.  Sizes: about
 * 3 N sizeof(T) + 3 ell N sizeof(T) bytes must fit (T = 4 mixed, 8 FP64), e.g.
 * ell = 10 and N <= 127,000 cells mixed or N <= 63,000 FP64; larger problems
 * are rejected with AAO_EINVAL and a message giving the bytes needed.
 *
 *   dim, n, kx, ky, kz, ell, alpha   as aao_create; face arrays, r and z must
 *                  be DEVICE pointers of the current device (or managed
 *                  memory); host pointers would need staging buffers, and
 *                  another GPU's memory is not reachable from the kernels:
 *                  both are rejected.
 *   prec, inner_its                  as aao_options.
 *   mu_max         > 1: upper spectral bound to use; 0: the Gershgorin bound.
 *   r, z           ell*N doubles each, block-major, distinct; r 8-byte and z
 *                  16-byte aligned (AAO_EINVAL otherwise: z is written two
 *                  doubles at a time and there is no staging buffer).
 *   stream         cudaStream_t for the work (NULL = default stream).
 *   err, err_len   optional buffer for a one-line message on failure.
 * The call synchronises the stream before returning.  On its first call on
 * a device it looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and caches it; make that first call before any
 * stream capture.  All calls on a device share the one array and it keeps
 * the last call's contents (the validity flag is cleared on every call), so
 * calls that overlap on the GPU -- from two host threads or two streams --
 * race and must be serialised by the caller.
 */
int aao_precond_apply_noalloc(int dim, const int64_t n[3], const double* kx, const double* ky,
                              const double* kz, int ell, double alpha, int prec, int inner_its,
                              double mu_max, const double* r, double* z, void* stream, char* err,
                              int err_len);

/* Release the handle and all workspace.  NULL is allowed. */
void aao_destroy(aao_handle h);

#ifdef __cplusplus
}
#endif

#endif /* AAO_H */
