/*
 * ssqcd -- contour-integral (Sakurai-Sugiura) eigensolver with shifted CG for
 * the Hermitian Wilson fermion matrix A = gamma5 (I - kappa D), on one GPU.
 *
 * C ABI.  Plain pointers and sizes only.  Every function returns an int
 * status (SSQCD_OK = 0 or one of the SSQCD_ERR_* codes below) and never
 * aborts; ssqcd_last_error() returns a thread-local message for the last
 * failure on the calling thread.
 *
 * Conventions used by every entry point:
 *  - lattice dims[4] = {X, Y, Z, T}; site s = x + X*(y + Y*(z + Z*t)),
 *    V = X*Y*Z*T, vector length n = 12 V;
 *  - complex numbers are interleaved (re, im) doubles ("complex128");
 *  - a spinor field is [V][4 spin][3 colour] complex128; a block of L fields
 *    is [L][V][4][3];
 *  - a gauge field is [4 mu][V][3][3] complex128, U[mu][s] is the link from
 *    s to s + mu_hat (mu = 0..3 = x, y, z, t), row-major 3x3;
 *  - the operator (Section 4 of the paper; D written out as the standard
 *    Wilson hopping matrix with r = 1):
 *      (D psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                        + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu),
 *    DeGrand-Rossi (chiral) gamma basis, gamma5 = gamma1 gamma2 gamma3 gamma4
 *    = diag(1, 1, -1, -1); periodic in x, y, z, sign bc_t on hops across
 *    the t boundary;
 *  - pointer arguments tagged "host or device" are read/written as device
 *    memory when the matching on_device flag is nonzero, else as host memory;
 *    the library copies what it needs and never keeps a caller's pointer.
 *
 * Ownership: handles own all device memory they allocate; destroy them with
 * the matching *_destroy.  All device work is issued on the CUDA stream given
 * at lattice creation; calls that return host data synchronise that stream.
 */
#ifndef SSQCD_H
#define SSQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SSQCD_OK            0
#define SSQCD_ERR_ARG       1  /* invalid argument (sizes, NULL, state)          */
#define SSQCD_ERR_OOM       2  /* device allocation failed                       */
#define SSQCD_ERR_BREAKDOWN 3  /* seed CG breakdown: |(p, K p)| < 1e-30 (r, r)   */
#define SSQCD_ERR_NOCONV    4  /* shifted CG hit max_iter before every shift met tol,
                               or a device-side wait hit its time limit (1 s)   */
#define SSQCD_ERR_CUDA      5  /* a CUDA runtime call failed                     */

/* ---- precision of the solve loop ------------------------------------------ */
#define SSQCD_FP64  0  /* everything in FP64 ("plain")                          */
#define SSQCD_MIXED 1  /* FP32 stencil + shift updates with FP16 12-parameter
                          links, FP64 reliable updates of the seed residual,
                          FP64 moments and Rayleigh-Ritz                       */
#define SSQCD_MIXED_F32LINKS 2  /* as SSQCD_MIXED with FP32 12-parameter links */
#define SSQCD_FP64_SHIFT32 3    /* FP64 links, stencil and seed recurrence; the
                                   per-shift vectors y and p-hat in FP32       */
#define SSQCD_FP64_DFSHIFT 4    /* as SSQCD_FP64_SHIFT32 with y and p-hat in
                                   float-float (hi + lo FP32 pair, 48-bit
                                   significand) updated on the FP32 pipes      */
#define SSQCD_DF           5    /* links, stencil, seed and shift vectors all in
                                   float-float on the FP32 pipes, and so are
                                   the Rayleigh-Ritz basis (CGS2), A T and the
                                   projected matrix; recurrence scalars, moment
                                   sums, eigenvectors and residuals in FP64    */

/* ---- eigenvalue extraction from the moments ---------------------------------- */
#define SSQCD_EXTRACT_RR     0  /* Rayleigh-Ritz on span(S_hat) (Section 2.1): eigenpairs
                                   with residuals (default)                            */
#define SSQCD_EXTRACT_HANKEL 1  /* block Hankel pencil of mu_k = V^H s_hat_k, k < 2M
                                   (Section 2.1): eigenvalues only, no basis and no
                                   extra matvecs; accuracy limited by the conditioning
                                   of the Hankel matrix (~1e-5 relative measured on
                                   4^4, against ~1e-14 for Rayleigh-Ritz)             */

/* ---- contour shapes --------------------------------------------------------- */
#define SSQCD_PATH_LINES  0  /* L+-: z = gamma + rho (x +- i beta), Section 3      */
#define SSQCD_PATH_CIRCLE 1  /* C:  z = gamma + rho exp(2 pi i (j + 1/2)/N), Sec. 2.1 */

typedef struct ssqcd_lattice_s* ssqcd_lattice;
typedef struct ssqcd_result_s*  ssqcd_result;

/* Options of ssqcd_ss_solve.  Zero-initialise, then set what you need;
 * ssqcd_default_opts() fills the defaults named below. */
typedef struct {
  int    path;            /* SSQCD_PATH_LINES (default) or SSQCD_PATH_CIRCLE     */
  double beta;            /* L+- half gap in units of rho (Section 3); 0.3       */
  int    nprime;          /* N': even, 4 <= N' <= N; 0 selects N/2 (Section 3)   */
  double tol;             /* per-shift stop ||r_j|| / ||v|| <= tol; 1e-12 (Sec. 4) */
  double sigma;           /* real seed shift (Section 2.2); 0 as in Section 4    */
  int    max_iter;        /* cap on seed CG iterations; 100000                   */
  double rank_tol;        /* keep basis directions with singular value above
                             rank_tol * largest; 1e-14                           */
  const double* sources;  /* host or device: [L][V][4][3] complex128, required  */
  int    sources_on_device;
  int    reliable_every;  /* mixed precisions: period (iterations) of the FP64
                             reliable update of the seed residual; 0 (default)
                             disables it -- measured to degrade the shifted
                             solutions once ||r|| nears the operator error      */
  int    windows;         /* lines only: split [a, b] into this many adjacent
                             windows with the same N, rho, beta whose cores tile
                             [a, b]; neighbouring windows reuse all but N' - 2 of
                             their points (Section 3), so one shifted-CG run
                             solves N + (windows - 1)(N' - 2) points; 1 default */
  int    extract;         /* SSQCD_EXTRACT_RR (default) or SSQCD_EXTRACT_HANKEL      */
  double hankel_tol;      /* Hankel: keep eigen-directions of the (Hermitian
                             positive semidefinite) block Hankel matrix above
                             hankel_tol * its largest eigenvalue; 1e-12          */
  int    refine;          /* Rayleigh-Ritz: 0 (default) Ritz vectors; 1 refined
                             Ritz vectors -- for each accepted Ritz value theta
                             the unit vector x of span(S_hat) minimising
                             ||(A - theta) x|| (Jia's refined projection, not in
                             the paper), reported with its Rayleigh quotient;
                             of two refined vectors that overlap by more than
                             1/sqrt(2) (a spurious Ritz value lands on its
                             neighbour's eigenvector) the one with the larger
                             ||(A - theta) x|| is dropped                      */
  int    basis;           /* SSQCD_FP64 and SSQCD_DF solves: 1 (default) stores
                             every seed residual r_k and the shift coefficients
                             of every iteration instead of updating the shift
                             vectors; the moments are then formed once, from
                             the stored residuals (y_j = sum_k g_jk r_k, the
                             g_jk from a backward recurrence over the shift
                             coefficients).  0: y_j and p-hat_j are updated
                             every iteration.  Other precisions always update */
  double basis_max_bytes; /* device memory the stored residuals may take; 0 =
                             sixteen times what the shift vectors would take
                             (32 N L n bytes: up to 32 N iterations) or 4 GiB
                             if more, at most half the free device memory.  A solve that
                             reaches it forms y_j and p-hat_j from the stored
                             residuals and continues with the per-iteration
                             updates (the same eigenpairs, other rounding)     */
  int    source_block;    /* 0 (default): all L sources in one shifted-CG run.
                             B with 0 < B < L: the sources run in blocks of B,
                             one shifted-CG run per block, each block's moments
                             formed before the next block starts (the seed
                             recurrences of different sources are independent,
                             so the moments are the same); only B sources'
                             stored residuals or shift vectors are held at a
                             time -- what lets the stored-residual form of a
                             large lattice fit the device memory            */
  double converged_tol;   /* residual bound of stats.n_converged; 1e-8.  The
                             paper accepts Ritz values by position (Section 3),
                             so an accepted pair can be a spurious Ritz value of
                             the filtered noise (residual ~0.5 when M L exceeds
                             the eigenvalue count); ssqcd_ss_eigpairs returns
                             every accepted pair with its residual, and
                             n_converged counts those at or below this bound */
  int    block_streams;   /* with source blocks: how many blocks' shifted-CG runs
                             proceed at once, each on its own stream (default
                             1: one after another).  The runs share only the
                             links, so the latency-bound seed kernels of one
                             run fill the gaps of the other's stencil; the
                             stored residuals of that many blocks are held at
                             once (basis_max_bytes is split between them) and
                             every source's arithmetic is unchanged        */
} ssqcd_opts;

/* Counters of one solve.  Times are device milliseconds between CUDA events. */
typedef struct {
  int    iterations;      /* seed CG iterations that updated a shift (= the largest
                             per-shift count; the Krylov-basis loop may apply the
                             stencil once more after the last freeze, because it
                             reads the live count one iteration late)            */
  int    max_shift_iters; /* largest per-shift iteration count at freeze           */
  int    matvecs_rr;      /* extra stencil applications in Rayleigh-Ritz           */
  int    rank;            /* dimension of the orthonormal basis kept               */
  int    n_ritz;          /* Ritz values computed (= rank)                         */
  int    n_accepted;      /* Ritz values inside the accepted interval              */
  int    reliable_updates;/* FP64 seed-residual refreshes (mixed path)             */
  double ms_cg;           /* shifted-CG loop                                        */
  double ms_moments;      /* moment accumulation                                    */
  double ms_rr;           /* Rayleigh-Ritz, acceptance and residuals                */
  double gamma, rho;      /* the (first) window actually used                       */
  int    points;          /* distinct quadrature points solved                      */
  long long shift_updates;/* sum over (source, shift) of iterations before freezing:
                             each is one y / p-hat update of n elements            */
  /* Per-kernel device time of the shifted-CG loop, filled when kernel timing
   * is on (ssqcd_set_kernel_timing): CUDA events around every launch, on the
   * stream each kernel runs on, in one chunk of 16 iterations out of every 4
   * (the sums below cover those timed iterations only); zero otherwise.  The
   * shift update of one iteration runs on a second stream beside the stencil
   * and seed work of the next, so these times overlap. */
  int    timed;
  int    launches_update;   /* timed iterations that did work                    */
  double ms_k_stencil;      /* stencil q = K p with the (p, q) partials and alpha */
  double ms_k_seed;         /* seed update r -= alpha q, shift scalars, freezing  */
  double ms_k_scalars;      /* seed direction p = r + beta p                      */
  double ms_k_update;       /* fused multi-shift update (update form), or the
                               shift-scalar kernel beside the chain (Krylov-basis
                               form: opts.basis)                                  */
  long long timed_shift_updates; /* (source, shift) updates in the timed iterations */
  int    basis;           /* 1: moments from the stored seed residuals; 2: began
                             so and switched to shift-vector updates at the
                             memory cap; 0: shift-vector updates throughout    */
  double basis_bytes;     /* device memory the stored residuals took at most  */
  int    n_converged;     /* accepted pairs with residual <= opts.converged_tol
                             (Rayleigh-Ritz only; the Hankel extraction has no
                             residuals and reports 0)                         */
  int    real_moments;    /* 1: the moments were combined from the stored seed
                             residuals with real coefficients -- the points
                             and weights come in conjugate pairs (line pairs
                             about a real centre, Section 3), the seed's CG
                             scalars are real, so each pair's coefficients
                             are conjugate and sum to a real number; 0: complex
                             coefficients (circle points, shift-vector updates,
                             or SSQCD_REAL_MOMENTS=0 in the environment).
                             With real coefficients and FP64 residuals the
                             combination runs on the tensor cores: residuals
                             and coefficients are split exactly into seven
                             8-bit bf16 slices on power-of-two grids and the
                             slice products summed exactly, so the moments
                             lie within 2^-56 of the operand scales of the
                             FP64 sum (SSQCD_MOMENTS_TC=0 in the environment:
                             the FP64-pipe combination instead)              */
} ssqcd_stats;

/* ---- lattice / operator ---------------------------------------------------- */

/* Create a lattice of extents dims[4] with hopping parameter kappa and time
 * boundary sign bc_t (+1 periodic, -1 antiperiodic), for the given precision
 * (one of the precision codes above; ssqcd_ss_solve runs its loop in it); every extent must be >= 1 and V <= 2^27.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream) on which all later work runs.
 * The operator is Section 4's A = gamma5 (I - kappa D).  On success *out owns
 * the gauge storage (no field until ssqcd_upload_gauge). */
int ssqcd_create_lattice(const int dims[4], double kappa, int bc_t, int precision,
                         void* cuda_stream, ssqcd_lattice* out);

/* Copy a gauge field ([4][V][3][3] complex128, host or device) into the
 * lattice, converting it to the library's device layout (and to FP16
 * 12-parameter storage as well for SSQCD_MIXED).  The caller keeps ownership
 * of `links`.  Links are used as given (no unitarity check). */
int ssqcd_upload_gauge(ssqcd_lattice lat, const double* links, int on_device);

/* out = A in for nrhs spinor fields ([nrhs][V][4][3] complex128; in and out
 * both host, or both device, per on_device; they must not overlap).  A is
 * the Hermitian fermion matrix of Section 4, applied in FP64. */
int ssqcd_apply_H(ssqcd_lattice lat, const double* in, double* out, int nrhs, int on_device);

/* Same as ssqcd_apply_H with the mixed path's operator: links stored FP16
 * (SSQCD_MIXED) or FP32 (SSQCD_MIXED_F32LINKS) as their first two rows, the
 * third rebuilt as conj(row0 x row1) (exact for SU(3)); spinors and
 * arithmetic in FP32.  Input and output stay complex128 at the boundary.
 * On a SSQCD_DF lattice: links, spinors and arithmetic in float-float
 * (relative error ~1e-14).  Requires a lattice created with one of the two
 * mixed precisions or with SSQCD_DF. */
int ssqcd_apply_H_mixed(ssqcd_lattice lat, const double* in, double* out, int nrhs, int on_device);

void ssqcd_lattice_destroy(ssqcd_lattice lat);

/* ---- quadrature (host) -------------------------------------------------------- */

/* Quadrature points z[N] and weights w[N] (complex128, host) for a contour:
 *  - SSQCD_PATH_LINES (Section 3): N/2 equally spaced points per line, ends
 *    included, x_i = -1 + 2 i/(N/2 - 1); z_{2i} = gamma + rho (x_i + i beta)
 *    on L+, z_{2i+1} = gamma + rho (x_i - i beta) on L-;
 *  - SSQCD_PATH_CIRCLE (Section 2.1): z_j = gamma + rho exp(2 pi i (j+1/2)/N).
 * Weights are the solution of the Section 3 system
 *    sum_j w_j zeta_j^(k-1) = delta_{k0}, k = 0..N-1, zeta_j = (z_j - gamma)/rho,
 * in closed form w_j = -P(0)/P'(zeta_j), P(zeta) = prod_k (zeta - zeta_k)
 * (for C this is zeta_j / N, Section 2.1 normalised by rho).
 * N must be even and >= 4 (lines) or >= 1 (circle); rho > 0. */
int ssqcd_contour(int path, double gamma, double rho, double beta, int N, double* z, double* w);

/* ---- shifted CG (Section 2.2) ---------------------------------------------- */

/* Solve (z_j I - A) y_{l,j} = v_l for the N shifts z[N] (complex128, host) and
 * L sources v ([L][V][4][3] complex128, host or device per on_device) with one
 * CG recurrence per source on the seed matrix sigma I - A (sigma real) and the
 * shifted-CG recurrences (residual of shift j = xi_j times the seed residual).
 * A shift stops when |xi_j| ||r|| / ||v_l|| <= tol.  Outputs (host or device,
 * per on_device, each may be NULL): y [L][N][V][4][3] complex128;
 * iters [L][N] int, the iteration at which each shift stopped; xi [L][N]
 * complex128, its final xi.  *seed_iters (may be NULL) receives the number of
 * seed iterations.  precision is one of the precision codes above; the two
 * mixed ones need a lattice created with that code, the others run on any
 * lattice (reliable_every as in ssqcd_opts).
 * Returns SSQCD_ERR_BREAKDOWN or SSQCD_ERR_NOCONV when the loop cannot finish
 * (outputs then hold the last iterate). */
int ssqcd_shifted_cg(ssqcd_lattice lat, int N, const double* z, int L, const double* v,
                     int on_device, double sigma, double tol, int max_iter, int precision,
                     int reliable_every,
                     double* y, int* iters, double* xi, int* seed_iters);

/* ---- moments (Eq. 2) ------------------------------------------------------------ */

/* s_hat[l][k] = sum_j w_j zeta_j^k y[l][j] for k < M (Eq. 2), on the device,
 * FP64.  y: [L][N][V][4][3] complex128 and s_hat: [L][M][V][4][3] complex128,
 * both host or both device per on_device; w, zeta: [N] complex128 host. */
int ssqcd_moments(ssqcd_lattice lat, int N, int M, int L, const double* w, const double* zeta,
                  const double* y, double* s_hat, int on_device);

/* Allocation-free variant of ssqcd_moments for callers that cannot allocate
 * device memory when they need the moments -- programs that hand all
 * device memory to their own pool or arena up front (a framework's caching
 * allocator, a solver embedded in a larger simulation), or loops that must
 * run within a fixed memory budget.  The paper has no counterpart; it
 * computes the same s_hat[l][k] = sum_j w_j zeta_j^k y[l][j] as
 * ssqcd_moments.
 * y: device, [L][N][n] complex128; s_hat: device, [L][M][n] complex128
 * (any element order, the same for both; n = 12 V for spinor fields);
 * w, zeta: host, [N] complex128, read during the call and passed to the
 * device as kernel parameters; work is issued on cuda_stream and the call
 * does not wait for it.  No cudaMalloc/cudaFree or allocating library call:
 * the only scratch, the N x M coefficient table, lives in a fixed 64 KiB
 * device array held by every GPU that loads the library until exit, so
 * N * M <= 4096 and N <= 256 (else SSQCD_ERR_ARG).  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current and caches it for the process; do not call again on a
 * device whose context was destroyed (cudaDeviceReset).  All calls share
 * the array: calls that overlap on the GPU (different streams, no
 * ordering) race. */
int ssqcd_moments_noalloc(int N, int M, int L, long long n, const double* w, const double* zeta,
                          const double* y, double* s_hat, void* cuda_stream);

/* ---- the eigensolver --------------------------------------------------------------- */

void ssqcd_default_opts(ssqcd_opts* opts);

/* Find the eigenpairs of A in the accepted interval [interval[0], interval[1]]
 * (the paper's Sections 2-3): quadrature points on the line pair L+- placed so
 * that the N' central points span the interval (gamma = (a + b)/2,
 * rho = (b - a)/2 (N/2 - 1)/(N'/2 - 1)), or on the circle C of centre
 * (a + b)/2 and radius (b - a)/2; shifted CG for all N points and L sources;
 * moments s_hat_k, k < M; Rayleigh-Ritz on span(S_hat) (n x M L); Ritz values
 * in [a, b] are accepted.  With opts.windows = K > 1 (lines only) the
 * interval is tiled by K windows whose points are solved together in one
 * shifted-CG run; each window has its own moments and Rayleigh-Ritz and
 * accepts the Ritz values in its share [a_k, a_{k+1}) of [a, b].  With
 * opts.extract = SSQCD_EXTRACT_HANKEL the moments run to k < 2M (2M <= N)
 * and the eigenvalues come from the block Hankel pencil instead (eigenvalues
 * only: residuals NaN, no eigenvectors).  The lattice precision decides the
 * solve loop.
 * *out receives a result handle (even when the status is an error other than
 * SSQCD_ERR_ARG/OOM, so its stats can be read). */
int ssqcd_ss_solve(ssqcd_lattice lat, const double interval[2], int N, int M, int L,
                   const ssqcd_opts* opts, ssqcd_result* out);

/* Several windows out of one shifted-CG run: K intervals
 * intervals[k] = [a_k, b_k] (host, [K][2] doubles, any positions, e.g. on both
 * sides of the spectral gap around zero), each with its own quadrature
 * points placed as in ssqcd_ss_solve with one window (same N, N', beta and
 * path from opts) -- Section 3's windows, which the paper solves one after
 * another.  The points of all windows (exact duplicates merged) go into one
 * seed recurrence per source (Section 2.2: one Krylov space serves every
 * shift); each window then has its own moments s_hat_k, k < M (Eq. 2),
 * Rayleigh-Ritz (or Hankel) extraction, and accepts the Ritz values in its
 * own [a_k, b_k].  The result holds the accepted pairs of all windows sorted
 * by eigenvalue; stats.points counts the distinct points and stats.gamma /
 * stats.rho give the first window.  opts.windows must be 0 or 1.  Errors as
 * ssqcd_ss_solve. */
int ssqcd_ss_solve_windows(ssqcd_lattice lat, int K, const double* intervals, int N, int M, int L,
                           const ssqcd_opts* opts, ssqcd_result* out);

/* The filtered block of one window without the extraction: the shifted CG
 * of ssqcd_ss_solve (same options, same quadrature points, the same choice
 * between per-iteration shift-vector updates and the stored seed residuals,
 * opts.basis) and its moments s_hat_k = sum_j w_j zeta_j^k y_j, k < M (Eq. 2),
 * of the first window.  s_hat: [L][M][V][4][3] complex128, host or device
 * (s_hat_on_device), written by the library; stats (may be NULL) receives
 * the shifted-CG counters.  Errors as ssqcd_ss_solve. */
int ssqcd_ss_moments(ssqcd_lattice lat, const double interval[2], int N, int M, int L, const ssqcd_opts* opts,
                     double* s_hat, int s_hat_on_device, ssqcd_stats* stats);

/* Read a result.  *count receives the number of accepted eigenpairs; pass
 * evals = NULL first to query it.  evals [count] (ascending), residuals
 * [count] = ||A x - lambda x||_2 with ||x||_2 = 1 (Section 4), evecs
 * [count][V][4][3] complex128 (host; may be NULL; SSQCD_ERR_ARG if the solve
 * used the Hankel extraction, which has none), stats (may be NULL). */
int ssqcd_ss_eigpairs(ssqcd_result res, int* count, double* evals, double* evecs,
                      double* residuals, ssqcd_stats* stats);

void ssqcd_result_destroy(ssqcd_result res);

/* ---- request scheduler: many solves in flight on one GPU --------------------------- */

/* Continuous batching of independent eigen-window requests (each one
 * ssqcd_ss_solve, on any lattice), driven by one host thread.  A submitted
 * request waits in a FIFO; ssqcd_server_progress admits requests from its
 * head while the estimated device memory of the running ones (dominated by
 * the N x L shift vectors, or by the stored seed residuals up to the
 * request's cap -- the cap ssqcd_ss_solve would use, so that the result is
 * the same; a request that does not fit the budget with it runs the update
 * form) stays within the budget, runs every admitted request on its own
 * stream with its shifted-CG chunks enqueued ahead, so the kernels of all
 * running requests interleave on the device, and finishes each request
 * whose shifts have all frozen (moments, extraction, memory freed).  A
 * request's arithmetic does not depend on the others: its result is the
 * same alone and in the mix.  Not a part of the paper. */
typedef struct ssqcd_server_s* ssqcd_server;

#define SSQCD_REQ_QUEUED  0
#define SSQCD_REQ_RUNNING 1
#define SSQCD_REQ_DONE    2
#define SSQCD_REQ_FAILED  3

/* memory_budget: device bytes the running requests may hold (0: 80% of the
 * currently free memory). */
int ssqcd_server_create(size_t memory_budget, ssqcd_server* out);

/* Queue a request; arguments as ssqcd_ss_solve (the sources are copied now,
 * host or device).  *id receives its handle.  SSQCD_ERR_OOM if the request
 * alone needs more than the budget; SSQCD_ERR_ARG as ssqcd_ss_solve.  The
 * lattice must outlive the request. */
int ssqcd_server_submit(ssqcd_server srv, ssqcd_lattice lat, const double interval[2], int N, int M,
                        int L, const ssqcd_opts* opts, long long* id);

/* Queue a request for several windows out of one shifted-CG run; arguments
 * as ssqcd_ss_solve_windows.  With opts.source_block = B < L the request
 * runs its sources in blocks of B, one shifted-CG run after another (its
 * admission estimate counts one block's shift vectors or stored residuals
 * and the moments of all L sources).  Errors as ssqcd_server_submit. */
int ssqcd_server_submit_windows(ssqcd_server srv, ssqcd_lattice lat, int K, const double* intervals, int N, int M,
                                int L, const ssqcd_opts* opts, long long* id);

/* Admit, advance and finish requests.  wait = 0 never blocks on the device
 * (returns at once when all running work is still in flight); wait = 1
 * blocks until at least one running request could move.  *completed (may be
 * NULL) receives the number of requests finished (done or failed) by this
 * call. */
int ssqcd_server_progress(ssqcd_server srv, int wait, int* completed);

/* State (SSQCD_REQ_*) of a request and its latency so far or at completion
 * (ms from submission; may be NULL). */
int ssqcd_server_status(ssqcd_server srv, long long id, int* state, double* latency_ms);

/* Hand over a finished request's result (destroy it with
 * ssqcd_result_destroy) and forget the request; returns the request's own
 * status (its result handle, if any, is still handed over).  SSQCD_ERR_ARG
 * if the request is unknown or not finished. */
int ssqcd_server_take(ssqcd_server srv, long long id, ssqcd_result* out);

/* Device bytes the scheduler reserves for a request while it runs (its
 * admission estimate). */
int ssqcd_server_request_bytes(ssqcd_server srv, long long id, size_t* bytes);

/* Requests so far that waited at the head of the queue because the running
 * requests' memory left no room for them (each counted once). */
int ssqcd_server_deferred(ssqcd_server srv, long long* requests);

/* Number of requests queued, running and finished (not yet taken). */
int ssqcd_server_counts(ssqcd_server srv, int* queued, int* running, int* finished);

/* Waits for the running requests' device work and frees everything. */
void ssqcd_server_destroy(ssqcd_server srv);

/* ---- small dense helper (host) ----------------------------------------------------- */

/* Eigen-decomposition of an m x m complex Hermitian matrix (row-major
 * complex128, host; only the lower triangle is read): evals[m] ascending,
 * evecs[m][m] row-major with eigenvector k in column k (may be NULL).  This
 * is the small eigenproblem of the Rayleigh-Ritz step (Section 2.1);
 * Householder reduction to real tridiagonal form, then implicit symmetric
 * QR steps with Wilkinson shifts. */
int ssqcd_small_eigh(int m, const double* a, double* evals, double* evecs);

/* ---- diagnostics ------------------------------------------------------------------------- */

const char* ssqcd_last_error(void);

/* Device time of the stencil alone: `reps` applications of A (after two
 * warm-up applications) to nrhs device-resident fields, in the lattice's
 * precision (SSQCD_FP64 / _FP64_SHIFT32 / _FP64_DFSHIFT: FP64; SSQCD_DF:
 * float-float; the mixed ones: FP32 spinors with their 12-parameter links),
 * CUDA events on the lattice stream.  *ms_per_call receives the mean time of
 * one application (all nrhs fields). */
int ssqcd_time_stencil(ssqcd_lattice lat, int nrhs, int reps, double* ms_per_call);

/* The FP32 stencil of the mixed precisions (ssqcd_apply_H_mixed,
 * ssqcd_time_stencil) has six variants: 0/1 -- every rhs of a block of 32
 * sites, warp w applying direction w with its two links loaded once for all
 * rhs, at 4/3 blocks an SM; 2/3 -- one thread per site and pair of rhs, all
 * eight hops, at 4/3 blocks an SM; 4/5 -- the same with the two rhs in the
 * two lanes of the paired FP32 instructions (rhs-pair layout, converted
 * around the kernel; even nrhs only), at 4/3 blocks an SM.  By default (-1)
 * the first application for a given lattice volume, rhs count and link
 * storage times every variant (three launches each, CUDA events on the
 * lattice stream, skipped while the stream is being captured) and keeps the
 * fastest for that key; ssqcd_time_stencil times the chosen kernel alone.
 * ssqcd_set_stencil_variant(v) forces variant v (0..7; 4-7 fall back to 2-3
 * for an odd nrhs, 6-7 to 4-5 where the lattice's X does not divide 128 or
 * 128 / X does not divide Y) for later calls in this process, or returns to
 * tuning (-1); SSQCD_ERR_ARG otherwise.  Not a part of the paper: the paper's
 * operator (Section 4) is the same in every variant. */
int ssqcd_set_stencil_variant(int variant);

/* The tuning recorded for this lattice (created with SSQCD_MIXED or
 * SSQCD_MIXED_F32LINKS) and nrhs: *variant the chosen variant, us[8] (may be
 * NULL) the measured microseconds per application of each (0 for a variant
 * not timed).  SSQCD_ERR_ARG
 * if nothing was tuned for that key yet. */
int ssqcd_stencil_tuning(ssqcd_lattice lat, int nrhs, int* variant, double* us);

/* Kernel launches issued by this process so far (all entry points). */
long long ssqcd_kernel_launches(void);

/* Turn per-kernel CUDA-event timing of the shifted-CG loop on (1) or off (0)
 * for later solves in this process (see the ms_k_* fields of ssqcd_stats).
 * Timing adds two event records per timed launch. */
int ssqcd_set_kernel_timing(int enable);

#ifdef __cplusplus
}
#endif
#endif /* SSQCD_H */
