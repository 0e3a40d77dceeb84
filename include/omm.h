/*
 * omm.h -- C ABI of the GB300 library for the preconditioned orbital minimization method
 * (Lu & Yang, "Preconditioning orbital minimization method for planewave
 * discretization", arXiv:1603.09724).
 *
 * Problem (Sec. 1, eq. tracemin; Sec. 4 eq. ex1mat): H = -Delta/2 + V on the periodic box
 * [0, L)^d, discretised pseudospectrally on an m^d grid (kinetic symbol (2 pi^2/L^2)|k|^2,
 * k in [-m/2, m/2)^d), shifted by sigma so that H - sigma < 0.  The library minimises
 * E_omm(X) = 1/2 tr((2I - X^*X) X^*(H - sigma)X) (eq. omm) over X in C^{n x N} by the
 * preconditioned nonlinear CG of Algorithm 1 with an exact quartic line search; the
 * preconditioner is the pole expansion of the Fermi projector (Sec. 3.1, eqs. dFOP,
 * direct, lst): P R = sum_j w_j (H - sigma - z_j)^-1 R, each shifted system solved
 * roughly by restarted GMRES whose right preconditioner is the sparsifying
 * preconditioner of Sec. 3.2 (eqs. GLu, QG, P), set up once per pole on the host and
 * applied on the device by triangular solves.  Alternatively the preconditioner is the
 * precomputed U U^* of Sec. 3.3, Algorithm 2 (omm_build_projector), or, for comparison,
 * one of the Fourier-diagonal TPA-type preconditioners of Sec. 2.2 (omm_set_gtpa).
 *
 * Layout conventions
 *   - A grid function is n = m^d contiguous complex values, x index fastest
 *     (flat index x + m*(y + m*z)), real/imaginary interleaved.
 *   - A block of N grid functions is column-major: column j at offset j*n.
 *   - Complex type: complex128 (two doubles) when the handle precision is OMM_FP64,
 *     complex64 (two floats) when it is OMM_MIXED.  V is always double on input.
 *   - Pointers documented as "device" must be CUDA device (or managed) memory of the
 *     current device; "host" pointers are ordinary host memory.
 * Ownership: inputs are copied or only read during the call; the handle owns all of its
 * device state and frees it in omm_destroy.  Device pointers passed in are borrowed
 * for the duration of the call.
 * Streams: every device operation is ordered on the stream given to omm_create.  The
 * triangular solves of different poles run on streams the handle owns (omm_params.
 * trsv_streams), forked from and joined back to that stream with events inside each call.
 * Calls that return host values (energies, statistics) synchronise that stream; the others
 * are asynchronous with respect to the host.
 * Threads: a handle must not be used by two threads at once.  No C++ exception crosses
 * this interface; every call returns an omm_status.
 */
#ifndef OMM_H
#define OMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct omm_ctx* omm_t;

typedef enum {
  OMM_OK = 0,
  OMM_EINVAL = -1,        /* invalid argument (null pointer, bad size, bad interval)    */
  OMM_ENOMEM = -2,        /* device or host allocation failed                            */
  OMM_EUNSUPPORTED = -3,  /* grid size / dimension / option not supported                */
  OMM_ENOTCONV = -4,      /* iteration limit reached (statistics are still filled)       */
  OMM_ETIMEOUT = -5,      /* a bounded device-side wait gave up                          */
  OMM_ECUDA = -6,         /* a CUDA runtime call failed (see omm_last_error_message)     */
  OMM_ESHIFT = -7,        /* H - sigma is not negative definite (E_omm unbounded below)  */
  OMM_ESTATE = -8         /* call out of order (e.g. iterate before poles are set)       */
} omm_status;

typedef enum { OMM_FP64 = 0, OMM_MIXED = 1 } omm_precision;

/* Right preconditioner of the GMRES pole solves. */
typedef enum {
  OMM_INNER_SPARSIFY = 0,  /* sparsifying preconditioner P^-1 Q G (Sec. 3.2)               */
  OMM_INNER_KINETIC = 1,   /* shifted kinetic inverse G = (T + <V> - sigma - z)^-1 (PP, Test 1) */
  OMM_INNER_NONE = 2       /* no preconditioner                                              */
} omm_inner;

typedef struct {
  int dim;         /* 2 or 3                                    */
  int m[3];        /* points per dimension (equal; 2^a 3^b)     */
  double box_len;  /* L: the box is [0, L)^dim                  */
} omm_grid;

typedef struct {
  int precision;        /* omm_precision                                               */
  int inner;            /* omm_inner                                                   */
  int gmres_m;          /* restart length (Sec. 4: 15), 1..15                          */
  int gmres_cycles;     /* maximum number of cycles (Sec. 4: 5)                        */
  double gmres_rtol;    /* relative residual tolerance per system (Sec. 4: 1e-5)      */
  int gmres_fixed;      /* 1: run every cycle to gmres_m steps (no tolerance test)     */
  int stencil_radius;   /* radius r of the (2r+1)^d sparsifying stencil (1)            */
  double pivot_floor;   /* static pivoting: pivots below pivot_floor*|row| are raised  */
  double tol;           /* CG stop: |E_{m+1} - E_m| <= tol |E_{m+1}| (Sec. 4: 1e-13)   */
  int maxit;            /* maximum CG iterations per round                             */
  int refilter;         /* extra (filter + CG) rounds after the first                  */
  int gram_tensor;      /* 1: complex64 Grams on tcgen05 tensor cores (TF32 x 3 split,
                           FP64 split-K sum); 0: CUDA cores.  FP64 handles use CUDA cores */
  int real_orbitals;    /* 1: X is kept real (H is real symmetric with the symmetric
                           kinetic symbol, and Sec. 3.1 writes the pole solutions
                           real).  omm_set_poles then folds each conjugate pair
                           (z, w), (conj z, conj w) into one solve:
                           w Y + conj(w Y) = 2 Re(w Y) for real right-hand sides, so the
                           pole expansion costs P/2 GMRES solves; poles must come in
                           conjugate pairs (or be real with real weight), else
                           omm_set_poles returns OMM_EINVAL.  omm_set_orbitals drops the
                           imaginary part of the block.  0: complex X, P solves.       */
  int trsv_streams;     /* streams for the triangular solves, one group of poles each
                           (1..8; 0 = 8: one pole per stream for the folded 16-pole
                           rule).  Several let the latency-bound top of the elimination
                           tree of one group overlap the other groups' work; use 1 when
                           many handles already run concurrently (serving).           */
  int trsv_persistent;  /* 1: the supernode heights of the triangular solves of all poles
                           run in one cooperative launch per application (grid barriers
                           between the phases, every wait bounded); 0 (default): one
                           launch per height and direction on trsv_streams streams,
                           which measured faster (the poles' heights overlap instead of
                           marching in step).  Keep 0 when several handles run at once
                           on one GPU (serving)                                         */
  int fixed_iters;      /* > 0: every CG round runs exactly this many iterations of
                           Algorithm 1 (no energy test; a fixed launch schedule for
                           timing and capture); 0: the energy criterion and maxit      */
  double refilter_rtol; /* GMRES tolerance of the rounds after the first (the refilter
                           and its CG iterations); 0: gmres_rtol.  The final subspace
                           error follows the GMRES tolerance of the last round, so a
                           tight value here buys the 1e-6 angle for a few applications */
  double gap;           /* lambda_{N+1} - lambda_N of H, if known (> 0): omm_solve then
                           reports the Davis-Kahan bound resid_orth / gap on the sine of
                           the largest principal angle to the exact invariant subspace;
                           0: not reported                                             */
  int launch_overlap;   /* 1 (default): the launches of the triangular solves are
                           programmatic dependent launches: each one is scheduled while
                           the one before it on its stream runs, loads its factor values
                           and index lists, and waits for that launch's results only
                           before it reads them; 0: ordinary launches                 */
  int device_factor;    /* 1 (default): omm_set_poles factors the sparsifying matrix P of
                           every pole on the device (multifrontal LU height by height,
                           all fronts of a height and all poles per launch, in the
                           handle's precision); the host computes only each pole's
                           stencil q (Sec. 3.2, eq. QG).  0: the host factorisation in
                           FP64 (rounded to the handle's precision), as before.  Grids
                           too small for the stencil use the host factorisation.       */
} omm_params;

typedef struct {
  int iters;               /* CG iterations done                                       */
  int filters;             /* filter applications (1 + refilter rounds run)            */
  int converged;           /* 1 if the energy criterion was met                        */
  double energy;           /* E_omm after the last step, from the iteration's Grams    */
  double energy_fp64;      /* E_omm recomputed in FP64 (omm_solve / omm_energy)        */
  double resid_fp64;       /* ||HX - X S^-1 K||_F / ||X||_F in FP64 (omm_solve)        */
  double gmres_relres_max; /* largest GMRES residual estimate of the last pole solve   */
  int gmres_iters_max;     /* largest GMRES step count of the last pole solve          */
  int gmres_iters_total;   /* sum of GMRES steps over all CG iterations (max per call) */
  double grad_norm;        /* ||Grad||_F of the last CG gradient (Sec. 2.1), FP64 sum   */
  double resid_orth;       /* ||H Q - Q (Q^* H Q)||_F with Q = X R^-1, S = R^* R the
                              Cholesky factor of X^* X: the residual of the orthonormal
                              basis of span X, FP64 on the device (omm_solve)           */
  double angle_bound;      /* resid_orth / omm_params.gap (sin theta theorem of Davis
                              and Kahan); 0 when no gap is given                        */
} omm_stats;

/* Human-readable text for a status code (static storage; no counterpart in the paper). */
const char* omm_strerror(omm_status s);
/* Text of the last CUDA failure or refusal reason recorded by this thread (static per-thread
 * storage; no counterpart in the paper). */
const char* omm_last_error_message(void);

/* Defaults: FP64, sparsifying inner preconditioner, GMRES(15) x 5 cycles, rtol 1e-5
 * (Sec. 4), stencil radius 1, pivot floor 1e-12, tol 1e-13, maxit 50, no refilter,
 * trsv_persistent 0, fixed_iters 0, refilter_rtol 0 (= gmres_rtol), gap 0 (no angle bound),
 * launch_overlap 1, device_factor 1.
 * Errors: OMM_EINVAL (p NULL). */
omm_status omm_default_params(omm_params* p);

/* Diagonal shift (Sec. 1): sigma = T_max + max(max V, 0) + 1e-3 (T_max + max V - min V),
 * T_max = (2 pi^2/L^2) sum_d (m/2)^2.  By Weyl's inequality H - sigma < 0.
 * V: host, n doubles.  Errors: OMM_EINVAL. */
omm_status omm_default_shift(const omm_grid* g, const double* V, double* shift);

/* Create a handle for H = -Delta/2 + V - sigma on the grid (Sec. 4 eq. ex1mat, shifted as in
 * Sec. 1).  V: host, n doubles, copied.  N: number of states (1 <= N < n).
 * shift: sigma; must exceed T_max + max V (else OMM_ESHIFT).  p: NULL for defaults.
 * stream: a cudaStream_t (NULL = legacy default stream).  Allocates the device work
 * space of the CG on the current device (the GMRES work space of the poles is allocated
 * by omm_set_poles; at most 32 poles).  All arguments are checked on the host before any
 * device work: OMM_EINVAL for a non-finite V or shift, NaN or negative tolerances or pivot
 * floor, or other parameters out of range.
 * Errors: OMM_EINVAL, OMM_EUNSUPPORTED (grid), OMM_ESHIFT, OMM_ENOMEM, OMM_ECUDA. */
omm_status omm_create(const omm_grid* g, const double* V, int N, double shift, const omm_params* p,
                      void* stream, omm_t* out);
void omm_destroy(omm_t h);

/* Pole rules (host helpers, no handle).  z, w: host, 2P doubles each (re, im pairs).
 *
 * omm_poles_fermi: quadrature of the contour integral of eq. FOP by the conformal map of
 * an annulus (Sec. 3.1, eq. dFOP): the strip 0 < Im u < K' is mapped by s = sn(u; k) and
 * a Moebius map onto the plane minus [a, b] (occupied: lam_1 .. lam_N, a may be any lower
 * bound) and [c, +inf) (unoccupied, c <= lam_{N+1}); P trapezoid nodes on Im u = K'/2.
 * Error decays like exp(-pi K' P / (4K)).  Needs a < b < c and P >= 2 even.
 * omm_poles_circle: trapezoid rule on |z - center| = radius (r(lam) = 1/(1+((lam-c)/R)^P)). */
omm_status omm_poles_fermi(double a, double b, double c, int P, double* z, double* w);
omm_status omm_poles_circle(double center, double radius, int P, double* z, double* w);

/* Set the pole expansion P R = sum_j w_j (H - sigma - z_j)^-1 R (eq. dFOP): z, w host,
 * 2P doubles each; 1 <= P <= 32.  With the sparsifying inner preconditioner this builds,
 * for every pole, the stencil row q (SVD of G(a, a^c), eq. QG), the sparse matrix P_j
 * (eq. P), its nested-dissection multifrontal LU (host, FP64) and uploads the factors.
 * With real_orbitals the conjugate pairs are folded first (see omm_params).  A projector
 * built by omm_build_projector no longer applies after new poles and is dropped.
 * Errors: OMM_EINVAL (P out of range, a non-finite z or w, an unpaired pole with
 * real_orbitals: the previous poles stay), OMM_ENOMEM, OMM_ECUDA (the handle then has no
 * poles until a later call succeeds: calls that need them return OMM_ESTATE). */
omm_status omm_set_poles(omm_t h, int P, const double* z, const double* w);

/* Copy the current orbitals X of eq. omm (the start of Algorithm 1) in (X: device, n x N,
 * handle precision) or out.
 * Errors: OMM_EINVAL (NULL handle or X), OMM_ECUDA. */
omm_status omm_set_orbitals(omm_t h, const void* X);
omm_status omm_get_orbitals(omm_t h, void* X);

/* Filter the orbitals once: X <- P X (Sec. 4: the starting guess is filtered) with the pole
 * expansion, or U U^* once a projector is built (never with gTPA).
 * Errors: OMM_ESTATE if no poles are set. */
omm_status omm_filter(omm_t h);

/* k steps of Algorithm 1 from the current X (restarting the CG: the first step uses the
 * steepest preconditioned direction).  st may be NULL.  Returns OMM_OK, or OMM_ESHIFT if
 * the quartic was not bounded below; OMM_ESTATE if neither poles nor gTPA are set;
 * OMM_ENOTCONV (st filled, fewer than k steps) if the energy, the line-search step or the
 * Polak-Ribiere beta became non-finite (numerical breakdown; the message says so). */
omm_status omm_iterate(omm_t h, int k, omm_stats* st);

/* Whole solve (Algorithm 1 with the filtered start of Sec. 4): filter, CG until the energy
 * criterion or maxit, then refilter rounds (GMRES at refilter_rtol),
 * then the FP64 check of the result on the device (with gTPA set: one CG round from the
 * given orbitals, no filter): X converted to complex128, FP64 H-apply and Grams
 * S = X^* X, K = X^* (H - sigma) X; one CTA computes E_omm = tr K - 1/2 tr(S K) (eq. omm),
 * the Cholesky factor S = R^* R, R^-1 and S^-1 K; FP64 block updates form the residuals
 * HX - X S^-1 K and (HX - X S^-1 K) R^-1 (stats energy_fp64, resid_fp64, resid_orth,
 * angle_bound).  Returns OMM_ENOTCONV (with st filled) if maxit was reached
 * in the last round or the CG broke down on a non-finite energy, step or beta (then no
 * further rounds run); OMM_ESTATE if neither poles nor gTPA are set. */
omm_status omm_solve(omm_t h, omm_stats* st);

/* The solve of omm_solve with a fixed schedule, enqueued on the handle's stream without
 * any host synchronisation, host copy or allocation, so that it can be captured in a CUDA
 * graph (stream capture) and replayed, alone or with the solves of other handles on
 * their own streams (no counterpart in the paper: the batched form of many Hamiltonians).
 * Needs fixed_iters > 0 (every CG round runs exactly that many iterations); every GMRES
 * cycle runs all gmres_m steps, and unless gmres_fixed = 1 the systems that meet the
 * tolerance are masked on the device from then on (their kernels return at once).  The
 * handle's work space must exist: call omm_solve once first.  The energy criterion is not tested (st->converged of omm_read_result
 * reports whether the last step met it).  Results stay on the device until
 * omm_read_result.
 * Errors: OMM_EINVAL (fixed_iters not set), OMM_ESTATE (no poles / gTPA, or no prior
 * omm_solve), OMM_ECUDA. */
omm_status omm_solve_enqueue(omm_t h);
/* Synchronises the handle's stream and returns the statistics of the last
 * omm_solve_enqueue (iterations, filters, energies, FP64 residuals, angle bound, GMRES
 * statistics of the last pole solve).
 * Errors: OMM_ESTATE (nothing enqueued), OMM_ESHIFT (the quartic was not bounded below),
 * OMM_ENOTCONV (a non-finite energy, step or beta), OMM_ETIMEOUT, OMM_ECUDA. */
omm_status omm_read_result(omm_t h, omm_stats* st);

/* E_omm (eq. omm) of the current X evaluated in FP64 (FP64 H-apply and FP64 Grams).
 * Errors: OMM_EINVAL (NULL handle or E), OMM_ENOMEM (first call allocates the FP64
 * work space), OMM_ECUDA. */
omm_status omm_energy(omm_t h, double* E);

/* ---- building blocks on caller buffers (the steps of one iteration) ------------ */

/* The pseudospectral H-apply (Sec. 4 eq. ex1mat), shifted as in eq. lst:
 * Y = (H - sigma - s) X for ncols columns: X, Y device, n x ncols, handle precision;
 * s = s_re + i s_im (pass s = -sigma for the unshifted -Delta/2 + V).
 * Errors: OMM_EINVAL (NULL pointers, ncols < 0), OMM_ENOMEM, OMM_ECUDA. */
omm_status omm_apply_h(omm_t h, const void* X, void* Y, int ncols, double s_re, double s_im);

/* The Gram blocks of eq. omm and Sec. 2.1 (X^*X, X^*HX, ...):
 * C = A^* B (na x nb, complex128, row-major, device, ldc = nb): A, B device blocks of
 * na and nb columns in the handle precision.
 * Errors: OMM_EINVAL (NULL pointers, na or nb < 1), OMM_ENOMEM, OMM_ECUDA, OMM_ETIMEOUT (a
 * bounded wait of the tensor-core Gram gave up; the flag stays set for the handle). */
omm_status omm_gram(omm_t h, const void* A, int na, const void* B, int nb, void* C);

/* Grad = 2 HX - X (X^*HX) - HX (X^*X) with H = H - sigma (Sec. 2.1): X device block of
 * N columns; HX and Grad device blocks (HX computed internally; may be NULL).
 * Errors: OMM_EINVAL (NULL handle, X or Grad), OMM_ENOMEM, OMM_ECUDA, OMM_ETIMEOUT. */
omm_status omm_gradient(omm_t h, const void* X, void* HX, void* Grad);

/* The exact line search of Algorithm 1 on eq. omm: quartic coefficients c[5] of
 * E_omm(X + tD) and its minimising step *t
 * (host outputs); X, D device blocks of N columns.
 * Errors: OMM_EINVAL (NULL handle, X or D), OMM_ECUDA, OMM_ETIMEOUT. */
omm_status omm_quartic(omm_t h, const void* X, const void* D, double* c, double* t);

/* Sparsifying preconditioner of pole j on ncols columns: U = P_j^-1 Q_j (G_j B)
 * (Sec. 3.2).  B, U device, handle precision.  Errors: OMM_ESTATE without poles or if
 * the inner preconditioner is not OMM_INNER_SPARSIFY. */
omm_status omm_precond_apply(omm_t h, int pole, const void* B, void* U, int ncols);

/* Pole-expansion preconditioner on N columns: Y = sum_j w_j Y_j with Y_j the GMRES
 * solution of (H - sigma - z_j) Y_j = R started from R (Sec. 3.1 eqs. direct, lst); with a
 * projector built (omm_build_projector), Y = U U^* R; with gTPA set (omm_set_gtpa), Y = P_t R.
 * R, Y device blocks of N columns.  st may be NULL (fills the gmres_* fields).
 * Errors: OMM_EINVAL (NULL pointers), OMM_ESTATE (neither poles nor gTPA set), OMM_ENOMEM,
 * OMM_ECUDA, OMM_ETIMEOUT. */
omm_status omm_pole_solve(omm_t h, const void* R, void* Y, omm_stats* st);

/* Precomputed preconditioner (Sec. 3.3, Algorithm 2): Y = sum_j w_j Y_j with
 * (H - sigma - z_j) Y_j = B solved by the handle's GMRES (started from B), U = an orthonormal
 * basis of N dominant columns of Y (rank-revealing step: Cholesky of Y^* Y with diagonal
 * pivoting, the Gram form of QR with column pivoting; then Cholesky QR; all in FP64, U
 * stored in the handle precision), and from then on the handle's preconditioner is U U^*
 * (omm_iterate, omm_filter, omm_solve, omm_pole_solve): one Gram U^* R and one block update
 * U (U^* R) per application instead of the pole solves.  Drops a gTPA preconditioner.
 * B: device, n x ncols, handle precision, a Gaussian block (real for real orbitals);
 * ncols = N (k = 0 extra columns, as in the paper's experiments) or 2N (k = N: the pivoting
 * then picks well-conditioned columns, which keeps the GMRES error of Y from being
 * amplified by the conditioning of a square random block).  Costs ncols / N pole solves.
 * st may be NULL (fills the gmres_* fields of the pole solves).
 * Errors: OMM_ESTATE without poles; OMM_EINVAL for another ncols or if Y is numerically
 * rank deficient (a Cholesky pivot <= 0). */
omm_status omm_build_projector(omm_t h, const void* B, int ncols, omm_stats* st);

/* Return to the pole-expansion preconditioner (Sec. 3.1) from U U^* (Sec. 3.3; frees
 * nothing; U is kept until the next
 * omm_build_projector or omm_destroy).
 * Errors: OMM_EINVAL (NULL handle). */
omm_status omm_drop_projector(omm_t h);

/* Fourier-diagonal comparison preconditioner of Sec. 2.2 (eqs. Lap, TPA, gTPA), the
 * TPA-type preconditioners the experiments of Sec. 4 compare against: the plane-wave
 * component k of R is multiplied by
 *     g_t(s) = p_t(s) / (p_t(s) + c_{t+1} s^{t+1}),  p_t(s) = c_0 + c_1 s + ... + c_t s^t,
 *     s = |k|^2 / tau, k the integer wave vector in [-m/2, m/2)^d.
 * t = 0 with c = (1, 1) is eq. Lap; t = 3 with c = (27, 18, 12, 8, 16) is eq. TPA.
 * c: host, t + 2 doubles (copied), all >= 0 with c_0 > 0 and c_{t+1} > 0; NULL selects
 * c_k = 27 (2/3)^k (k <= t), c_{t+1} = 3 * 27 (2/3)^{t+1}, which is eq. TPA at t = 3 (the
 * paper gives no coefficients for other t).  tau > 0: Sec. 4 takes the largest kinetic
 * energy (1/2) sum_k |k|^2 |xhat_j(k)|^2 over the normalised exact eigenvectors.  0 <= t <= 16.
 * While set, it is the handle's preconditioner (omm_iterate, omm_solve, omm_pole_solve; one
 * fused FFT / multiply / inverse-FFT pass per application), ahead of a projector or the pole
 * expansion, and omm_solve starts the CG from the orbitals as given (no filter step).
 * omm_filter keeps filtering with the pole expansion or the projector.  Poles are not needed.
 * Errors: OMM_EINVAL (t, c or tau out of range; a gTPA preconditioner already set stays),
 * OMM_ENOMEM, OMM_ECUDA (no gTPA preconditioner is then set). */
omm_status omm_set_gtpa(omm_t h, int t, const double* c, double tau);

/* Stop using the gTPA preconditioner of Sec. 2.2 (back to the projector or the pole
 * expansion).
 * Errors: OMM_EINVAL (NULL handle). */
omm_status omm_drop_gtpa(omm_t h);

/* Statistics of the sparsifying factor of pole j (Sec. 3.2; host outputs, any may be NULL):
 * number of supernodes, factor entries (L + U), smallest |pivot| / largest |pivot|,
 * number of perturbed pivots.
 * Errors: OMM_EINVAL (NULL handle, pole out of range), OMM_ESTATE (no poles, or the inner
 * preconditioner is not the sparsifying one). */
omm_status omm_factor_info(omm_t h, int pole, int* nsuper, long long* nnz, double* pivot_ratio, int* nperturbed);

/* C = A^* B like omm_gram, but without a handle and without allocating any device
 * memory (the paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc, e.g. code that runs inside another framework's memory manager which has
 * already reserved the device memory, or paths where the implicit synchronisation and
 * latency of cudaMalloc/cudaFree are not acceptable).
 * precision: OMM_FP64 (A, B complex128) or OMM_MIXED (complex64); A: n x na and B: n x nb,
 * device, column-major; C: na x nb complex128, row-major, device; stream: cudaStream_t.
 * The split-K partial sums live in a fixed 8 MiB device array compiled into the library
 * (524288 complex128 entries, held by every GPU that loads the library until the process
 * exits).  na * nb must not exceed 524288, else OMM_EINVAL (the message says why).
 * The first call on a device, with that device current, resolves the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's partials (every partial is
 * written before it is read, so nothing needs clearing): calls that overlap on the GPU
 * (different streams, or different host threads on one device) race and must be
 * serialised by the caller.  Asynchronous with respect to the host. */
omm_status omm_gram_noalloc(int precision, const void* A, int na, const void* B, int nb, size_t n, void* C,
                            void* stream);

/* Device allocator hook (no counterpart in the paper) used by subsequent omm_create calls
 * (NULL, NULL restores cudaMalloc/cudaFree).  alloc(bytes, ctx) returns device memory or
 * NULL.
 * Errors: OMM_EINVAL (exactly one of alloc and release is NULL). */
omm_status omm_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* ctx);

/* Bytes of device memory the handle holds (no counterpart in the paper).
 * Errors: OMM_EINVAL (NULL handle or bytes). */
omm_status omm_device_bytes(omm_t h, size_t* bytes);

/* ---- instrumentation (no counterpart in the paper; used to report roofline figures) --
 * Kernel classes: 0 happly (H-apply), 1 greenq (Green symbol + Q stencil), 2 trsv_levels
 * (sparsifying triangular solves above the leaves, L and U), 3 orth (GMRES Gram-Schmidt),
 * 4 gram, 5 block_update (gradient), 6 vector (axpby, dots, GMRES vector updates),
 * 7 small (line search, Givens, counters), 8 trsv_leaf (the leaves' L and U solves).  For every class the handle always counts
 * calls, kernels launched and algorithmic bytes moved; with profiling enabled it also
 * brackets each call with CUDA events on the handle's stream and sums the elapsed
 * milliseconds.  omm_profile_enable(h, 1) resets the counters and turns the events on;
 * omm_profile_enable(h, 2) resets the counters with the events off (counting only, no
 * timing overhead); omm_profile_enable(h, 0) turns the events off.  omm_profile_read
 * synchronises the stream.  omm_profile_class_name returns NULL for an unknown class.
 * Algorithmic bytes of the triangular solves (classes 2 and 8): 4 complex values per
 * unknown and active system (right-hand side in, y out, y in, x out) plus every pole's
 * factor once per application; omm_profile_read_impl returns the implementation's own
 * byte model of the class (the update rows, assembled separator right-hand sides and
 * boundary gathers included), equal to the algorithmic bytes for the other classes.
 * Errors: OMM_EINVAL (NULL handle or output, class or mode out of range). */
omm_status omm_profile_enable(omm_t h, int on);
omm_status omm_profile_read(omm_t h, int cls, long long* calls, long long* kernels, double* ms, double* bytes);
omm_status omm_profile_read_impl(omm_t h, int cls, double* impl_bytes);
/* Algorithmic real flops counted for a class since the last omm_profile_enable: the
 * supernode products of the triangular solves (class 2: 8 flops per W_f or W_b entry of a
 * pole and active system of that pole, Sec. 3.2's dense supernode blocks); 0 for the
 * classes whose bound is memory traffic.  Errors: OMM_EINVAL (NULL handle or output, class
 * out of range). */
omm_status omm_profile_read_flops(omm_t h, int cls, double* flops);
const char* omm_profile_class_name(int cls);

#ifdef __cplusplus
}
#endif

#endif /* OMM_H */
