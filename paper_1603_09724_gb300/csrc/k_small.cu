// N x N algebra in FP64 on one CTA: quartic coefficients of E_omm(X + tD), the exact
// line search, energies, the Grams of the updated X, and the Polak-Ribiere beta.
//
// eq. omm: E(X) = 1/2 tr((2I - X^*X)(X^*HX)).  With S(t) = A + tB + t^2 C and
// K(t) = A_H + t B_H + t^2 C_H (A = X^*X, B = X^*D + D^*X, C = D^*D and the same with H)
// E(t) = tr K(t) - 1/2 tr(S(t) K(t)) = c0 + c1 t + ... + c4 t^4.  The minimiser over real
// t is one of the real roots of E'(t) (a cubic); c4 = -1/2 tr(C C_H) > 0 for H < 0.
// H = H0 - sigma: the Grams come from the unshifted H0 X (so that no large shift enters
// the working-precision data) and sigma is applied here in FP64.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace omm {

namespace {

__device__ double cubic_value(const double* a, double t) { return ((a[3] * t + a[2]) * t + a[1]) * t + a[0]; }
__device__ double cubic_deriv(const double* a, double t) { return (3.0 * a[3] * t + 2.0 * a[2]) * t + a[1]; }

// Real roots of a[3] t^3 + a[2] t^2 + a[1] t + a[0] (a[3] != 0); returns the count.
// Depressed cubic y^3 + P y + Q = 0 with t = y - p2/3; Cardano for one real root,
// the trigonometric form for three; each root is refined by Newton steps.
__device__ int cubic_real_roots(const double* a, double* r) {
  const double p2 = a[2] / a[3], p1 = a[1] / a[3], p0 = a[0] / a[3];
  const double P = p1 - p2 * p2 / 3.0;
  const double Q = 2.0 * p2 * p2 * p2 / 27.0 - p2 * p1 / 3.0 + p0;
  const double disc = 0.25 * Q * Q + P * P * P / 27.0;
  int nr = 0;
  if (disc > 0.0) {
    const double sq = sqrt(disc);
    const double u = cbrt(-0.5 * Q - copysign(sq, Q));
    const double y = (u != 0.0) ? u - P / (3.0 * u) : 0.0;
    r[nr++] = y - p2 / 3.0;
  } else if (P == 0.0) {
    r[nr++] = -p2 / 3.0;
  } else {
    const double mP = -P / 3.0;
    const double rad = sqrt(mP);
    double arg = -0.5 * Q / (mP * rad);
    arg = fmax(-1.0, fmin(1.0, arg));
    const double phi = acos(arg);
    const double twopi3 = 2.0943951023931954923084289221863353;  // 2 pi / 3
    for (int k = 0; k < 3; ++k) r[nr++] = 2.0 * rad * cos(phi / 3.0 - twopi3 * k) - p2 / 3.0;
  }
  for (int i = 0; i < nr; ++i) {
    double t = r[i];
    for (int it = 0; it < 4; ++it) {
      const double d = cubic_deriv(a, t);
      if (d == 0.0) break;
      const double step = cubic_value(a, t) / d;
      t -= step;
      if (fabs(step) <= 1e-16 * fabs(t)) break;
    }
    r[i] = t;
  }
  return nr;
}

__device__ double quartic(const double* c, double t) { return c[0] + t * (c[1] + t * (c[2] + t * (c[3] + t * c[4]))); }

template <int NV>
__device__ void block_sum_vec(double (&v)[NV], double* sh /* >= 32 * NV */) {
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid * NV + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sh[w * NV + q];
      v[q] = s;
    }
  }
  __syncthreads();
}

}  // namespace

// The fused Gram's blocks, shifted by sigma where H enters, as functions of (i, j).
struct LsBlocks {
  const double2* Cg;
  int N, ld;
  double sigma;
  __device__ double2 at(int r, int c) const { return Cg[(size_t)r * ld + c]; }
  __device__ double2 A(int i, int j) const { return at(i, j); }
  __device__ double2 B(int i, int j) const {
    const double2 a = at(i, N + j), b = at(N + i, j);
    return make_double2(a.x + b.x, a.y + b.y);
  }
  __device__ double2 Cm(int i, int j) const { return at(N + i, N + j); }
  __device__ double2 AH(int i, int j) const {
    const double2 h = at(i, 2 * N + j), s = at(i, j);
    return make_double2(h.x - sigma * s.x, h.y - sigma * s.y);
  }
  __device__ double2 BH(int i, int j) const {
    const double2 h1 = at(i, 3 * N + j), h2 = at(N + i, 2 * N + j), s = B(i, j);
    return make_double2(h1.x + h2.x - sigma * s.x, h1.y + h2.y - sigma * s.y);
  }
  __device__ double2 CH(int i, int j) const {
    const double2 h = at(N + i, 3 * N + j), s = at(N + i, N + j);
    return make_double2(h.x - sigma * s.x, h.y - sigma * s.y);
  }
};

// Line search in three launches (the traces are O(N^2) FP64 work that one CTA would run on
// one SM): ls_traces, one CTA per row i, sums row i's terms of the 12 traces
//   v: 0 trAH, 1 trBH, 2 trCH, 3 tr(A AH), 4 tr(A BH), 5 tr(B AH), 6 tr(A CH), 7 tr(B BH),
//      8 tr(C AH), 9 tr(B CH), 10 tr(C BH), 11 tr(C CH)
// into work[i][12]; ls_solve adds the rows in order, forms the quartic and finds its
// minimiser; ls_matrices forms M1, M2 at the chosen step.
constexpr int LS_NV = 12;

__global__ void __launch_bounds__(128) ls_traces_kernel(LsBlocks g, int have_d, double* __restrict__ work) {
  __shared__ double sh[32 * LS_NV];
  const int i = blockIdx.x, N = g.N;
  auto rmul = [](double2 p, double2 q) { return p.x * q.x - p.y * q.y; };  // Re(p q)
  double v[LS_NV];
#pragma unroll
  for (int q = 0; q < LS_NV; ++q) v[q] = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double2 a_ij = g.A(i, j), ah_ji = g.AH(j, i);
    if (i == j) v[0] += ah_ji.x;
    v[3] += rmul(a_ij, ah_ji);
    if (have_d) {
      const double2 b_ij = g.B(i, j), c_ij = g.Cm(i, j);
      const double2 bh_ji = g.BH(j, i), ch_ji = g.CH(j, i);
      if (i == j) {
        v[1] += bh_ji.x;
        v[2] += ch_ji.x;
      }
      v[4] += rmul(a_ij, bh_ji);
      v[5] += rmul(b_ij, ah_ji);
      v[6] += rmul(a_ij, ch_ji);
      v[7] += rmul(b_ij, bh_ji);
      v[8] += rmul(c_ij, ah_ji);
      v[9] += rmul(b_ij, ch_ji);
      v[10] += rmul(c_ij, bh_ji);
      v[11] += rmul(c_ij, ch_ji);
    }
  }
  block_sum_vec<LS_NV>(v, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < LS_NV; ++q) work[(size_t)i * LS_NV + q] = v[q];
}

__global__ void ls_solve_kernel(int N, int have_d, double tol, const double* __restrict__ work, OmmScalars* sc) {
  __shared__ double v[LS_NV];
  if (threadIdx.x < LS_NV) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += work[(size_t)i * LS_NV + threadIdx.x];   // rows in order
    v[threadIdx.x] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double c[5];
  c[0] = v[0] - 0.5 * v[3];
  c[1] = v[1] - 0.5 * (v[4] + v[5]);
  c[2] = v[2] - 0.5 * (v[6] + v[7] + v[8]);
  c[3] = -0.5 * (v[9] + v[10]);
  c[4] = -0.5 * v[11];
  double t = 0.0;
  int bad = 0;
  if (have_d) {
    if (!(c[4] > 0.0)) {
      bad = 1;
    } else {
      double a[4] = {c[1], 2.0 * c[2], 3.0 * c[3], 4.0 * c[4]};
      double r[3];
      const int nr = cubic_real_roots(a, r);
      double best = quartic(c, r[0]);
      t = r[0];
      for (int k = 1; k < nr; ++k) {
        const double e = quartic(c, r[k]);
        const double tie = 4.0 * 2.220446049250313e-16 * fmax(1.0, fabs(best));
        if (e < best - tie || (fabs(e - best) <= tie && fabs(r[k]) < fabs(t))) {
          best = e;
          t = r[k];
        }
      }
    }
  }
  for (int q = 0; q < 5; ++q) sc->c[q] = c[q];
  sc->t = t;
  sc->t_c = make_double2(t, 0.0);
  sc->one_c = make_double2(1.0, 0.0);
  sc->E0 = c[0];
  sc->E1 = quartic(c, t);
  sc->bad = bad;
  sc->converged = fabs(sc->E1 - sc->E0) <= tol * fabs(sc->E1);
}

// Grams of X + tD (unshifted K0), then M1 = -(K0 + 2 sigma (I - S)), M2 = -S
template <typename T>
__global__ void ls_matrices_kernel(LsBlocks g, int have_d, const OmmScalars* __restrict__ sc, cx_t<T>* __restrict__ M1,
                                   cx_t<T>* __restrict__ M2) {
  const int N = g.N;
  const double t = sc->t, sigma = g.sigma;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * N; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, j = idx % N;
    double2 S = g.A(i, j);
    double2 K0 = g.at(i, 2 * N + j);
    if (have_d) {
      const double2 b = g.B(i, j), cc = g.Cm(i, j);
      const double2 h1 = g.at(i, 3 * N + j), h2 = g.at(N + i, 2 * N + j), hd = g.at(N + i, 3 * N + j);
      S.x += t * b.x + t * t * cc.x;
      S.y += t * b.y + t * t * cc.y;
      K0.x += t * (h1.x + h2.x) + t * t * hd.x;
      K0.y += t * (h1.y + h2.y) + t * t * hd.y;
    }
    const double id = (i == j) ? 1.0 : 0.0;
    const double m1r = -(K0.x + 2.0 * sigma * (id - S.x));
    const double m1i = -(K0.y - 2.0 * sigma * S.y);
    M1[idx] = mk<cx_t<T>>((T)m1r, (T)m1i);
    M2[idx] = mk<cx_t<T>>((T)(-S.x), (T)(-S.y));
  }
}

cudaError_t launch_line_search(bool dbl, const double2* C, int N, double sigma, int have_d, double tol,
                               OmmScalars* sc, void* M1, void* M2, double* work, cudaStream_t st) {
  if (N < 1 || !work) return cudaErrorInvalidValue;
  const LsBlocks g{C, N, 4 * N, sigma};
  ls_traces_kernel<<<N, 128, 0, st>>>(g, have_d, work);
  ls_solve_kernel<<<1, 32, 0, st>>>(N, have_d, tol, work, sc);
  const int blocks = std::min((N * N + 255) / 256, 1024);
  if (dbl)
    ls_matrices_kernel<double><<<blocks, 256, 0, st>>>(g, have_d, sc, (double2*)M1, (double2*)M2);
  else
    ls_matrices_kernel<float><<<blocks, 256, 0, st>>>(g, have_d, sc, (float2*)M1, (float2*)M2);
  return cudaGetLastError();
}

__global__ void pr_beta_kernel(OmmScalars* sc, int first) {
  double beta = 0.0;
  if (!first && sc->ggp != 0.0) beta = (sc->gg - sc->gdot) / sc->ggp;
  sc->beta = beta;
  sc->beta_c = make_double2(beta, 0.0);
  sc->ggp = sc->gg;
}

cudaError_t launch_pr_beta(OmmScalars* sc, int first, cudaStream_t st) {
  pr_beta_kernel<<<1, 1, 0, st>>>(sc, first);
  return cudaGetLastError();
}

}  // namespace omm

namespace omm {

// M = scale * C for an N x N FP64 Gram C (row stride ldc), in the working precision
template <typename T>
__global__ void gram_to_matrix_kernel(const double2* __restrict__ C, int ldc, int N, double scale,
                                      cx_t<T>* __restrict__ M) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * N; idx += gridDim.x * blockDim.x) {
    const double2 c = C[(size_t)(idx / N) * ldc + idx % N];
    M[idx] = mk<cx_t<T>>((T)(scale * c.x), (T)(scale * c.y));
  }
}

cudaError_t launch_gram_to_matrix(bool dbl, const double2* C, int ldc, int N, double scale, void* M, cudaStream_t st) {
  const int blocks = (N * N + 255) / 256 < 1024 ? (N * N + 255) / 256 : 1024;
  if (dbl)
    gram_to_matrix_kernel<double><<<blocks, 256, 0, st>>>(C, ldc, N, scale, (double2*)M);
  else
    gram_to_matrix_kernel<float><<<blocks, 256, 0, st>>>(C, ldc, N, scale, (float2*)M);
  return cudaGetLastError();
}

}  // namespace omm

namespace omm {

// ---- FP64 check of a result (once per solve).  From the FP64 Gram C = X^*[X  (H - sigma) X]
// (N x 2N, row stride ldc): S = C[:, 0:N], K = C[:, N:2N].  One CTA:
//   E_omm = tr K - 1/2 tr(S K)                              (eq. omm)
//   S = R^* R (right-looking Cholesky, R upper), then R^-1 by back substitution, one
//   column per thread.
// The N x N arrays R, Rinv live in global memory (row-major); every step that reads what
// other threads wrote follows a __syncthreads, which orders global memory within the CTA.
// ok[0] = 0 if a pivot of S is not positive (X rank deficient), else 1.
__global__ void __launch_bounds__(1024) fp64_chol_kernel(const double2* __restrict__ Cg, int ldc, int N,
                                                          double* __restrict__ E, double2* R, double2* Rinv,
                                                          int* __restrict__ ok) {
  __shared__ double sh[32 * 2];
  __shared__ double dj;
  __shared__ int good;
  const int tid = threadIdx.x, bd = blockDim.x;
  double v[2] = {0.0, 0.0};
  for (int idx = tid; idx < N * N; idx += bd) {
    const int i = idx / N, j = idx % N;
    const double2 s = Cg[(size_t)i * ldc + j], k = Cg[(size_t)j * ldc + N + i];
    if (i == j) v[0] += Cg[(size_t)i * ldc + N + i].x;
    v[1] += s.x * k.x - s.y * k.y;
    R[idx] = (j >= i) ? s : make_double2(0.0, 0.0);
  }
  block_sum_vec<2>(v, sh);
  if (tid == 0) {
    *E = v[0] - 0.5 * v[1];
    good = 1;
  }
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (tid == 0) {
      const double d = R[(size_t)j * N + j].x;
      if (!(d > 0.0)) good = 0;
      dj = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    for (int k = j + tid; k < N; k += bd) {
      const double2 r = R[(size_t)j * N + k];
      R[(size_t)j * N + k] = (k == j) ? make_double2(dj, 0.0) : make_double2(r.x / dj, r.y / dj);
    }
    __syncthreads();
    const int m = N - j - 1;
    for (int e = tid; e < m * m; e += bd) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k < i) continue;
      const double2 a = R[(size_t)j * N + i], b = R[(size_t)j * N + k];   // conj(a) * b
      double2& t = R[(size_t)i * N + k];
      t.x -= a.x * b.x + a.y * b.y;
      t.y -= a.x * b.y - a.y * b.x;
    }
    __syncthreads();
  }
  for (int c = tid; c < N; c += bd) {
    for (int r = c + 1; r < N; ++r) Rinv[(size_t)r * N + c] = make_double2(0.0, 0.0);
    Rinv[(size_t)c * N + c] = make_double2(1.0 / R[(size_t)c * N + c].x, 0.0);
    for (int r = c - 1; r >= 0; --r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = r + 1; k <= c; ++k) {
        const double2 a = R[(size_t)r * N + k], b = Rinv[(size_t)k * N + c];
        acc.x += a.x * b.x - a.y * b.y;
        acc.y += a.x * b.y + a.y * b.x;
      }
      const double d = R[(size_t)r * N + r].x;
      Rinv[(size_t)r * N + c] = make_double2(-acc.x / d, -acc.y / d);
    }
  }
  if (tid == 0) *ok = good;
}

// Out = scale * op(A) B for N x N complex double matrices (row-major, row strides lda, ldb,
// N for Out); op(A) = A^* when CT.  One thread per output entry.
template <bool CT>
__global__ void zgemm_small_kernel(const double2* __restrict__ A, int lda, const double2* __restrict__ B, int ldb,
                                   double2* __restrict__ Out, int N, double scale) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int i = idx / N, j = idx % N;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < N; ++k) {
    const double2 a = CT ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k];
    const double2 b = B[(size_t)k * ldb + j];
    if (CT) {   // conj(a) b
      acc.x += a.x * b.x + a.y * b.y;
      acc.y += a.x * b.y - a.y * b.x;
    } else {
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
  }
  Out[idx] = make_double2(scale * acc.x, scale * acc.y);
}

cudaError_t launch_fp64_check_small(const double2* C, int ldc, int N, double* E, double2* R, double2* Rinv,
                                    double2* T, double2* Mneg, int* ok, cudaStream_t st) {
  fp64_chol_kernel<<<1, 1024, 0, st>>>(C, ldc, N, E, R, Rinv, ok);
  const int nb = (N * N + 255) / 256;
  // T = R^-* K, then -S^-1 K = -R^-1 T  (S^-1 = R^-1 R^-*)
  zgemm_small_kernel<true><<<nb, 256, 0, st>>>(Rinv, N, C + N, ldc, T, N, 1.0);
  zgemm_small_kernel<false><<<nb, 256, 0, st>>>(Rinv, N, T, N, Mneg, N, -1.0);
  return cudaGetLastError();
}

}  // namespace omm
