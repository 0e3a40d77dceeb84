// Internal kernel launchers (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace omm {

// ---- k_fft.cu: fused shared-memory pseudospectral kernels
bool fused_fft_supported(int dim, int m, bool dbl);
cudaError_t launch_happly(bool dbl, int dim, int m, const void* X, void* Y, int ncols, const void* V,
                          const double2* shifts, int cols_per_group, const void* tw, double kin_over_n,
                          const int* active, cudaStream_t st);
// iperm: NULL (natural-order output) or n indices: out[iperm[i]] receives grid point i
cudaError_t launch_greenq(bool dbl, int dim, int m, const void* B, void* Out, int ncols, const void* ghat,
                          const void* q, int nq, int cols_per_group, const void* tw, const int* active,
                          const int* iperm, cudaStream_t st);

// ---- k_fft_big.cu: multi-pass (per-axis) kernels for large grids; tmp: ncols * n complex
bool big_fft_supported(int dim, int m);
// kernels one multi-pass H-apply (greenq = false) or Green apply (true) launches
int big_fft_launches(int dim, int m, bool dbl, bool greenq);
cudaError_t launch_happly_big(bool dbl, int dim, int m, const void* X, void* Y, int ncols, const void* V,
                              const double2* shifts, int cols_per_group, const void* tw, double kin_over_n,
                              const int* active, void* tmp, cudaStream_t st);
cudaError_t launch_greenq_big(bool dbl, int dim, int m, const void* B, void* Out, int ncols, const void* ghat,
                              const void* q, int nq, int cols_per_group, const void* tw, const int* active,
                              const int* iperm, void* tmp, cudaStream_t st);

// ---- k_blas.cu
// C (na x nb, complex double, row-major, ldc) = A^H B; A, B column blocks of length n (lda = ldb = n).
// work: at least gram_work_bytes(na, nb, n) bytes.
size_t gram_work_bytes(int na, int nb, size_t n);
cudaError_t launch_gram(bool dbl, const void* A, int na, const void* B, int nb, size_t n, double2* C, int ldc,
                        void* work, cudaStream_t st);
// ---- k_gram_tc.cu: the same Gram on tcgen05 tensor cores (complex64 inputs, TF32 x 3 split,
// FP32 accumulation in tensor memory, FP64 split-K sum).  err: device flag set to 1 if a
// bounded wait gave up.
bool gram_tc_supported(size_t n);
size_t gram_tc_work_bytes(int na, int nb, size_t n);
cudaError_t launch_gram_tc(const void* A, int na, const void* B, int nb, size_t n, double2* C, int ldc, void* work,
                           int* err, cudaStream_t st);
// Out = a*A + b*B + A*M1 + B*M2 (A, B: n x N blocks; M1, M2: N x N complex, working precision,
// row-major, in device memory; a, b real).
cudaError_t launch_block_update(bool dbl, const void* A, const void* B, const void* M1, const void* M2,
                                double a, double b, int N, size_t n, void* Out, cudaStream_t st);
// Y[i] = alpha * X[i] + beta * Y[i] over count complex elements; alpha, beta complex from
// device pointers (nullptr means 1 for alpha, 0 for beta).
cudaError_t launch_axpby(bool dbl, size_t count, const double2* alpha, const void* X, const double2* beta,
                         void* Y, cudaStream_t st);
// out[j] = sum over ncols of Re<A_j, B_j> partials -> result (double) written to *res (deterministic).
cudaError_t launch_redot(bool dbl, size_t count, const void* A, const void* B, double* res, void* work,
                         cudaStream_t st);
size_t redot_work_bytes();
// Convert block precision (count complex elements).
cudaError_t launch_convert(bool to_dbl, size_t count, const void* src, void* dst, cudaStream_t st);
// x <- Re(x) for count complex entries (imaginary parts set to zero)
cudaError_t launch_real_part(bool dbl, size_t count, void* x, cudaStream_t st);

// ---- k_small.cu: N x N algebra on one CTA (FP64)
struct OmmScalars {
  double c[5];        // quartic coefficients of E(X + tD)
  double t;           // line-search step
  double E0, E1;      // energy before / after the step
  double beta;        // Polak-Ribiere beta
  double gg, ggp;     // <G_m, G_m>, <G_{m-1}, G_{m-1}>
  double gdot;        // <G_m, G_{m-1}>
  double grad2;       // ||Grad||_F^2 of the last gradient
  double2 t_c;        // t as complex (for axpby)
  double2 beta_c;     // beta as complex
  double2 one_c;
  int converged;
  int bad;            // nonzero if the quartic was not bounded below
};
// From the fused Gram C = [X D]^H [X D HX HD] (2N x 4N, ldc = 4N; HX = H0 X unshifted):
// quartic coefficients with H = H0 - sigma, exact line search, energies; then the Grams of
// X + tD (S, K0) and the update matrices M1 = -(K0 + 2 sigma (I - S)), M2 = -S in the
// working precision for the next gradient.  If have_d == 0 only E0 and M1, M2 at t = 0.
// work: N x 12 doubles of device scratch (the per-row partial traces).
cudaError_t launch_line_search(bool dbl, const double2* C, int N, double sigma, int have_d, double tol,
                               OmmScalars* sc, void* M1, void* M2, double* work, cudaStream_t st);
// beta = (gg - gdot) / ggp (Polak-Ribiere); first == 1 sets beta = 0.
// M = scale * C (N x N FP64 Gram with row stride ldc) in the working precision
cudaError_t launch_gram_to_matrix(bool dbl, const double2* C, int ldc, int N, double scale, void* M, cudaStream_t st);
cudaError_t launch_pr_beta(OmmScalars* sc, int first, cudaStream_t st);
// FP64 check (one CTA + two small products): from C = X^*[X (H - sigma)X] (N x 2N, ldc)
// *E = E_omm, R (N x N) the Cholesky factor of S = X^*X (S = R^* R, upper), Rinv = R^-1,
// T work, Mneg = -S^-1 K; *ok = 0 if S is not positive definite.  All FP64, row-major.
cudaError_t launch_fp64_check_small(const double2* C, int ldc, int N, double* E, double2* R, double2* Rinv,
                                    double2* T, double2* Mneg, int* ok, cudaStream_t st);

// ---- k_krylov.cu: batched restarted GMRES over S systems of length n
struct KrylovDims {
  int S;            // systems
  int N;            // columns per pole (system s = p * N + c, rhs column c)
  size_t n;         // vector length
  int m;            // restart length
};
// r_s = b_c - (H0 b_c - shift_p b_c) for cycle 0 (x = b), from Hb = H0 b; writes V0 = r/|r|,
// beta, g0, active flags (relres > rtol unless fixed).
cudaError_t launch_krylov_init0(bool dbl, KrylovDims d, const void* b, const void* Hb, const double2* shifts,
                                void* V0, void* x, double* beta, double2* g, double* bnorm, int* active,
                                double rtol, int fixed, cudaStream_t st);
// r_s = b_c - Ax_s (Ax given), restart
cudaError_t launch_krylov_restart(bool dbl, KrylovDims d, const void* b, const void* Ax, void* V0, double* beta,
                                  double2* g, const double* bnorm, int* active, double rtol, int fixed,
                                  cudaStream_t st);
// CGS2 of w against V_0..V_k; writes V_{k+1} = w / h_{k+1,k}, h column k.
cudaError_t launch_krylov_orth(bool dbl, KrylovDims d, int k, void* V, void* w, double2* H, const int* active,
                               cudaStream_t st);
// Givens update of column k, residual estimate, deactivation; steps[s] = k+1 for active s.
cudaError_t launch_krylov_givens(KrylovDims d, int k, double2* H, double2* cs, double2* g, const double* bnorm,
                                 int* active, int* steps, double* est, double rtol, int fixed, int* nactive,
                                 cudaStream_t st);
// y = R^-1 g per system (steps[s] columns), x_s += Z y.
// itot[s] += steps[s].
cudaError_t launch_krylov_update(bool dbl, KrylovDims d, const double2* H, const double2* g, const int* steps,
                                 double2* y, const void* Z, void* x, int* itot, cudaStream_t st);
// *nactive = number of s with active[s] != 0
cudaError_t launch_count_active(KrylovDims d, const int* active, int* nactive, cudaStream_t st);
// out_c = sign * sum_p w_p x_{p N + c}
// out = sign * sum_p w_p x_p over the P poles; real_part: out = (Re(...), 0)
cudaError_t launch_pole_combine(bool dbl, KrylovDims d, int P, const double2* w, double sign, int real_part,
                                const void* x, void* out, cudaStream_t st);

}  // namespace omm
