// Batched restarted GMRES for the P x N shifted systems (H - sigma - z_p) y = b_c of the
// pole expansion (Sec. 3.1 eqs. direct / lst): right preconditioning, initial guess = the
// right-hand side, classical Gram-Schmidt with one re-orthogonalisation, Givens rotations
// on the small Hessenberg matrix, and the preconditioned basis Z kept for the update
// x += Z y.  One CTA per system for the vector work; one thread per system for the
// small (m <= 16) dense work.  System s = p * N + c.
#include <cstdint>
#include <initializer_list>

#include "common.cuh"
#include "kernels.h"

namespace omm {

constexpr int KMAX = 16;   // max basis size (restart m <= 15)
constexpr int KT = 256;    // threads per system CTA

namespace {

template <int NV>
__device__ void block_reduce(double (&v)[NV], double* sh) {
  // sh: >= NV * (KT / 32) doubles; result broadcast to all threads
#pragma unroll
  for (int q = 0; q < NV; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * (KT / 32) + wid] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < KT / 32; ++w) s += sh[q * (KT / 32) + w];
    v[q] = s;
  }
}

}  // namespace

// ------------------------------------------------------------------ cycle start
template <typename T>
__global__ void __launch_bounds__(KT) krylov_init_kernel(KrylovDims d, const cx_t<T>* __restrict__ b,
                                                         const cx_t<T>* __restrict__ Hx, const double2* __restrict__ shifts,
                                                         cx_t<T>* __restrict__ V0, cx_t<T>* __restrict__ x,
                                                         double* __restrict__ beta, double2* __restrict__ g,
                                                         double* __restrict__ bnorm, int* __restrict__ active,
                                                         double rtol, int fixed, int first) {
  using C = cx_t<T>;
  __shared__ double sh[2 * (KT / 32)];
  const int s = blockIdx.x;
  const int c = s % d.N, p = s / d.N;
  const C* bc = b + (size_t)c * d.n;
  // first cycle: Hx = H0 b_c (one per column), x = b, Ax = H0 b - shift_p b
  // later cycles: Hx = A x_s (per system)
  const C* hx = first ? Hx + (size_t)c * d.n : Hx + (size_t)s * d.n;
  const double2 sh_p = first ? shifts[p] : make_double2(0.0, 0.0);
  const T sr = (T)sh_p.x, si = (T)sh_p.y;
  T a0 = 0, a1 = 0;
  for (size_t i = threadIdx.x; i < d.n; i += KT) {
    const C bi = bc[i];
    C r = csub(bi, hx[i]);
    if (first) {  // + shift * b
      r.x += sr * bi.x - si * bi.y;
      r.y += sr * bi.y + si * bi.x;
      x[(size_t)s * d.n + i] = bi;
    }
    a0 += r.x * r.x + r.y * r.y;
    a1 += bi.x * bi.x + bi.y * bi.y;
  }
  double acc[2] = {(double)a0, (double)a1};
  block_reduce<2>(acc, sh);
  const double bt = sqrt(acc[0]);
  const double bn = first ? sqrt(acc[1]) : bnorm[s];
  const T inv = bt > 0.0 ? (T)(1.0 / bt) : T(0);
  for (size_t i = threadIdx.x; i < d.n; i += KT) {
    const C bi = bc[i];
    C r = csub(bi, hx[i]);
    if (first) {
      r.x += sr * bi.x - si * bi.y;
      r.y += sr * bi.y + si * bi.x;
    }
    V0[(size_t)s * d.n + i] = cscale(r, inv);
  }
  if (threadIdx.x == 0) {
    beta[s] = bt;
    if (first) bnorm[s] = bn;
    for (int k = 0; k <= d.m; ++k) g[(size_t)s * (KMAX + 1) + k] = make_double2(k == 0 ? bt : 0.0, 0.0);
    const double rel = bn > 0.0 ? bt / bn : 0.0;
    active[s] = (bt > 0.0) && (fixed || rel > rtol);
  }
}

// The same cycle start for complex64 with an even grid and 16-byte aligned vectors: two
// entries per float4 load / store.
__global__ void __launch_bounds__(KT) krylov_init_c64x2_kernel(KrylovDims d, const float4* __restrict__ b,
                                                               const float4* __restrict__ Hx,
                                                               const double2* __restrict__ shifts,
                                                               float4* __restrict__ V0, float4* __restrict__ x,
                                                               double* __restrict__ beta, double2* __restrict__ g,
                                                               double* __restrict__ bnorm, int* __restrict__ active,
                                                               double rtol, int fixed, int first) {
  __shared__ double sh[2 * (KT / 32)];
  const int s = blockIdx.x;
  const int c = s % d.N, p = s / d.N;
  const size_t n2 = d.n / 2;
  const float4* bc = b + (size_t)c * n2;
  const float4* hx = first ? Hx + (size_t)c * n2 : Hx + (size_t)s * n2;
  const double2 sh_p = first ? shifts[p] : make_double2(0.0, 0.0);
  const float sr = (float)sh_p.x, si = (float)sh_p.y;
  auto resid = [&](float2 bi, float2 hi) {   // b - A x (first: b - (H0 b - shift b))
    float2 r = csub(bi, hi);
    if (first) {
      r.x += sr * bi.x - si * bi.y;
      r.y += sr * bi.y + si * bi.x;
    }
    return r;
  };
  float a0 = 0, a1 = 0;
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 bv = bc[i], hv = hx[i];
    const float2 b0 = make_float2(bv.x, bv.y), b1 = make_float2(bv.z, bv.w);
    const float2 r0 = resid(b0, make_float2(hv.x, hv.y)), r1 = resid(b1, make_float2(hv.z, hv.w));
    if (first) x[(size_t)s * n2 + i] = bv;
    a0 += r0.x * r0.x + r0.y * r0.y + r1.x * r1.x + r1.y * r1.y;
    a1 += b0.x * b0.x + b0.y * b0.y + b1.x * b1.x + b1.y * b1.y;
  }
  double acc[2] = {(double)a0, (double)a1};
  block_reduce<2>(acc, sh);
  const double bt = sqrt(acc[0]);
  const double bn = first ? sqrt(acc[1]) : bnorm[s];
  const float inv = bt > 0.0 ? (float)(1.0 / bt) : 0.f;
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 bv = bc[i], hv = hx[i];
    const float2 r0 = resid(make_float2(bv.x, bv.y), make_float2(hv.x, hv.y));
    const float2 r1 = resid(make_float2(bv.z, bv.w), make_float2(hv.z, hv.w));
    V0[(size_t)s * n2 + i] = make_float4(r0.x * inv, r0.y * inv, r1.x * inv, r1.y * inv);
  }
  if (threadIdx.x == 0) {
    beta[s] = bt;
    if (first) bnorm[s] = bn;
    for (int k = 0; k <= d.m; ++k) g[(size_t)s * (KMAX + 1) + k] = make_double2(k == 0 ? bt : 0.0, 0.0);
    const double rel = bn > 0.0 ? bt / bn : 0.0;
    active[s] = (bt > 0.0) && (fixed || rel > rtol);
  }
}

static bool pairs_ok(const KrylovDims& d, std::initializer_list<const void*> ptrs) {
  if (d.n % 2) return false;
  for (const void* q : ptrs)
    if (q && (uintptr_t)q % 16) return false;
  return true;
}

cudaError_t launch_krylov_init0(bool dbl, KrylovDims d, const void* b, const void* Hb, const double2* shifts, void* V0,
                                void* x, double* beta, double2* g, double* bnorm, int* active, double rtol, int fixed,
                                cudaStream_t st) {
  if (dbl)
    krylov_init_kernel<double><<<d.S, KT, 0, st>>>(d, (const double2*)b, (const double2*)Hb, shifts, (double2*)V0,
                                                   (double2*)x, beta, g, bnorm, active, rtol, fixed, 1);
  else if (pairs_ok(d, {b, Hb, V0, x}))
    krylov_init_c64x2_kernel<<<d.S, KT, 0, st>>>(d, (const float4*)b, (const float4*)Hb, shifts, (float4*)V0,
                                                 (float4*)x, beta, g, bnorm, active, rtol, fixed, 1);
  else
    krylov_init_kernel<float><<<d.S, KT, 0, st>>>(d, (const float2*)b, (const float2*)Hb, shifts, (float2*)V0,
                                                  (float2*)x, beta, g, bnorm, active, rtol, fixed, 1);
  return cudaGetLastError();
}

cudaError_t launch_krylov_restart(bool dbl, KrylovDims d, const void* b, const void* Ax, void* V0, double* beta,
                                  double2* g, const double* bnorm, int* active, double rtol, int fixed,
                                  cudaStream_t st) {
  if (dbl)
    krylov_init_kernel<double><<<d.S, KT, 0, st>>>(d, (const double2*)b, (const double2*)Ax, nullptr,
                                                   (double2*)V0, nullptr, beta, g, (double*)bnorm, active, rtol,
                                                   fixed, 0);
  else if (pairs_ok(d, {b, Ax, V0}))
    krylov_init_c64x2_kernel<<<d.S, KT, 0, st>>>(d, (const float4*)b, (const float4*)Ax, nullptr, (float4*)V0,
                                                 nullptr, beta, g, (double*)bnorm, active, rtol, fixed, 0);
  else
    krylov_init_kernel<float><<<d.S, KT, 0, st>>>(d, (const float2*)b, (const float2*)Ax, nullptr,
                                                  (float2*)V0, nullptr, beta, g, (double*)bnorm, active, rtol, fixed,
                                                  0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ CGS2
// Classical Gram-Schmidt with one re-orthogonalisation of w against V_0..V_{KK-1}
// (KK = k + 1 is a template parameter so that the per-thread partial sums and basis
// values stay in registers).  Three sweeps over the basis:
//   1: h1 = V^H w
//   2: w' = w - V h1 (on the fly), h2 = V^H w', |w'|^2
//   3: w'' = w - V (h1 + h2), written as V_{k+1} = w'' / |w''| with
//      |w''|^2 = |w'|^2 - |h2|^2 (w'' is orthogonal to V, which is orthonormal).
template <typename T, int KK>
__global__ void __launch_bounds__(KT) krylov_orth_kernel(KrylovDims d, cx_t<T>* __restrict__ V,
                                                         const cx_t<T>* __restrict__ w, double2* __restrict__ H,
                                                         const int* __restrict__ active) {
  using C = cx_t<T>;
  constexpr int k = KK - 1;
  // loop unroll over the grid: more independent loads in flight when the basis is short
  constexpr int UF = KK <= 2 ? 4 : (KK <= 6 ? 2 : 1);
  __shared__ double sh[(2 * KK + 1) * (KT / 32)];
  const int s = blockIdx.x;
  if (!active[s]) return;
  const size_t n = d.n;
  const size_t vs = (size_t)d.S * n;   // stride between basis vectors
  const C* ws = w + (size_t)s * n;
  const C* Vs = V + (size_t)s * n;
  double h[2 * KK + 1];
  C ht[KK];
  C h1c[KK];
  // sweep 1
#pragma unroll
  for (int q = 0; q < KK; ++q) ht[q] = mk<C>(0, 0);
#pragma unroll UF
  for (size_t i = threadIdx.x; i < n; i += KT) {
    const C wi = ws[i];
#pragma unroll
    for (int j = 0; j < KK; ++j) ht[j] = cfmac(Vs[j * vs + i], wi, ht[j]);
  }
#pragma unroll
  for (int q = 0; q < KK; ++q) { h[2 * q] = (double)ht[q].x; h[2 * q + 1] = (double)ht[q].y; }
  h[2 * KK] = 0.0;
  block_reduce<2 * KK + 1>(h, sh);
  double h1[2 * KK];
#pragma unroll
  for (int q = 0; q < 2 * KK; ++q) h1[q] = h[q];
#pragma unroll
  for (int j = 0; j < KK; ++j) h1c[j] = mk<C>((T)h1[2 * j], (T)h1[2 * j + 1]);
  // sweep 2
#pragma unroll
  for (int q = 0; q < KK; ++q) ht[q] = mk<C>(0, 0);
  T nw = 0;
#pragma unroll UF
  for (size_t i = threadIdx.x; i < n; i += KT) {
    C wi = ws[i];
    C vv[KK];
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      vv[j] = Vs[j * vs + i];
      wi = csub(wi, cmul(h1c[j], vv[j]));
    }
#pragma unroll
    for (int j = 0; j < KK; ++j) ht[j] = cfmac(vv[j], wi, ht[j]);
    nw += wi.x * wi.x + wi.y * wi.y;
  }
#pragma unroll
  for (int q = 0; q < KK; ++q) { h[2 * q] = (double)ht[q].x; h[2 * q + 1] = (double)ht[q].y; }
  h[2 * KK] = (double)nw;
  block_reduce<2 * KK + 1>(h, sh);
  double h2sq = 0.0;
#pragma unroll
  for (int q = 0; q < 2 * KK; ++q) {
    h2sq += h[q] * h[q];
    h1[q] += h[q];
  }
  const double hn = sqrt(fmax(h[2 * KK] - h2sq, 0.0));
  const T inv = hn > 0.0 ? (T)(1.0 / hn) : T(0);
#pragma unroll
  for (int j = 0; j < KK; ++j) h1c[j] = mk<C>((T)h1[2 * j], (T)h1[2 * j + 1]);
  // sweep 3
  C* vk1 = V + (size_t)(k + 1) * vs + (size_t)s * n;
#pragma unroll UF
  for (size_t i = threadIdx.x; i < n; i += KT) {
    C wi = ws[i];
#pragma unroll
    for (int j = 0; j < KK; ++j) wi = csub(wi, cmul(h1c[j], Vs[j * vs + i]));
    vk1[i] = cscale(wi, inv);
  }
  if (threadIdx.x == 0) {
    double2* Hs = H + (size_t)s * (KMAX + 1) * KMAX;
    for (int j = 0; j <= k; ++j) Hs[j * KMAX + k] = make_double2(h1[2 * j], h1[2 * j + 1]);
    Hs[(k + 1) * KMAX + k] = make_double2(hn, 0.0);
  }
}

// The same CGS2 for complex64 bases with an even grid size: every thread moves two
// consecutive complex values per 16-byte load (float4), so twice the bytes are in flight
// per instruction on the three streaming sweeps.
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

template <int KK>
__global__ void __launch_bounds__(KT) krylov_orth_c64x2_kernel(KrylovDims d, float2* __restrict__ V,
                                                               const float2* __restrict__ w, double2* __restrict__ H,
                                                               const int* __restrict__ active) {
  using C = float2;
  constexpr int k = KK - 1;
  __shared__ double sh[(2 * KK + 1) * (KT / 32)];
  const int s = blockIdx.x;
  if (!active[s]) return;
  const size_t n2 = d.n / 2;
  const size_t vs2 = (size_t)d.S * n2;   // stride between basis vectors, in pairs
  const float4* ws = reinterpret_cast<const float4*>(w) + (size_t)s * n2;
  const float4* Vs = reinterpret_cast<const float4*>(V) + (size_t)s * n2;
  double h[2 * KK + 1];
  C ht[KK];
  C h1c[KK];
  // sweep 1: h1 = V^H w
#pragma unroll
  for (int q = 0; q < KK; ++q) ht[q] = mk<C>(0, 0);
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 wi = ws[i];
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      const float4 v = Vs[j * vs2 + i];
      ht[j] = cfmac(hi2(v), hi2(wi), cfmac(lo2(v), lo2(wi), ht[j]));
    }
  }
#pragma unroll
  for (int q = 0; q < KK; ++q) { h[2 * q] = (double)ht[q].x; h[2 * q + 1] = (double)ht[q].y; }
  h[2 * KK] = 0.0;
  block_reduce<2 * KK + 1>(h, sh);
  double h1[2 * KK];
#pragma unroll
  for (int q = 0; q < 2 * KK; ++q) h1[q] = h[q];
#pragma unroll
  for (int j = 0; j < KK; ++j) h1c[j] = mk<C>((float)h1[2 * j], (float)h1[2 * j + 1]);
  // sweep 2: w' = w - V h1 on the fly, h2 = V^H w', |w'|^2
#pragma unroll
  for (int q = 0; q < KK; ++q) ht[q] = mk<C>(0, 0);
  float nw = 0;
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 wi = ws[i];
    C wa = lo2(wi), wb = hi2(wi);
    float4 vv[KK];
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      vv[j] = Vs[j * vs2 + i];
      wa = csub(wa, cmul(h1c[j], lo2(vv[j])));
      wb = csub(wb, cmul(h1c[j], hi2(vv[j])));
    }
#pragma unroll
    for (int j = 0; j < KK; ++j) ht[j] = cfmac(hi2(vv[j]), wb, cfmac(lo2(vv[j]), wa, ht[j]));
    nw += wa.x * wa.x + wa.y * wa.y + wb.x * wb.x + wb.y * wb.y;
  }
#pragma unroll
  for (int q = 0; q < KK; ++q) { h[2 * q] = (double)ht[q].x; h[2 * q + 1] = (double)ht[q].y; }
  h[2 * KK] = (double)nw;
  block_reduce<2 * KK + 1>(h, sh);
  double h2sq = 0.0;
#pragma unroll
  for (int q = 0; q < 2 * KK; ++q) {
    h2sq += h[q] * h[q];
    h1[q] += h[q];
  }
  const double hn = sqrt(fmax(h[2 * KK] - h2sq, 0.0));
  const float inv = hn > 0.0 ? (float)(1.0 / hn) : 0.f;
#pragma unroll
  for (int j = 0; j < KK; ++j) h1c[j] = mk<C>((float)h1[2 * j], (float)h1[2 * j + 1]);
  // sweep 3: V_{k+1} = (w - V (h1 + h2)) / |w''|
  float4* vk1 = reinterpret_cast<float4*>(V) + (size_t)(k + 1) * vs2 + (size_t)s * n2;
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 wi = ws[i];
    C wa = lo2(wi), wb = hi2(wi);
#pragma unroll
    for (int j = 0; j < KK; ++j) {
      const float4 v = Vs[j * vs2 + i];
      wa = csub(wa, cmul(h1c[j], lo2(v)));
      wb = csub(wb, cmul(h1c[j], hi2(v)));
    }
    vk1[i] = make_float4(wa.x * inv, wa.y * inv, wb.x * inv, wb.y * inv);
  }
  if (threadIdx.x == 0) {
    double2* Hs = H + (size_t)s * (KMAX + 1) * KMAX;
    for (int j = 0; j <= k; ++j) Hs[j * KMAX + k] = make_double2(h1[2 * j], h1[2 * j + 1]);
    Hs[(k + 1) * KMAX + k] = make_double2(hn, 0.0);
  }
}

template <typename T>
static cudaError_t orth_dispatch(KrylovDims d, int k, void* V, void* w, double2* H, const int* active,
                                 cudaStream_t st) {
  using C = cx_t<T>;
#define ORTH_CASE(KK_)                                                                                   \
  case KK_:                                                                                              \
    krylov_orth_kernel<T, KK_><<<d.S, KT, 0, st>>>(d, (C*)V, (const C*)w, H, active);                    \
    break;
  // complex64 with an even grid: paired loads, up to 10 basis vectors (beyond, the paired
  // kernel needs more than 128 registers and would halve the CTAs per SM)
  if (sizeof(C) == sizeof(float2) && d.n % 2 == 0 && k + 1 <= 10 && (uintptr_t)V % 16 == 0 &&
      (uintptr_t)w % 16 == 0) {
#define ORTH2_CASE(KK_)                                                                                  \
  case KK_:                                                                                              \
    krylov_orth_c64x2_kernel<KK_><<<d.S, KT, 0, st>>>(d, (float2*)V, (const float2*)w, H, active);       \
    break;
    switch (k + 1) {
      ORTH2_CASE(1) ORTH2_CASE(2) ORTH2_CASE(3) ORTH2_CASE(4) ORTH2_CASE(5) ORTH2_CASE(6) ORTH2_CASE(7)
      ORTH2_CASE(8) ORTH2_CASE(9) ORTH2_CASE(10)
      default: return cudaErrorInvalidValue;
    }
#undef ORTH2_CASE
    return cudaGetLastError();
  }
  switch (k + 1) {
    ORTH_CASE(1) ORTH_CASE(2) ORTH_CASE(3) ORTH_CASE(4) ORTH_CASE(5) ORTH_CASE(6) ORTH_CASE(7) ORTH_CASE(8)
    ORTH_CASE(9) ORTH_CASE(10) ORTH_CASE(11) ORTH_CASE(12) ORTH_CASE(13) ORTH_CASE(14) ORTH_CASE(15)
    default: return cudaErrorInvalidValue;
  }
#undef ORTH_CASE
  return cudaGetLastError();
}

cudaError_t launch_krylov_orth(bool dbl, KrylovDims d, int k, void* V, void* w, double2* H, const int* active,
                               cudaStream_t st) {
  if (k < 0 || k + 1 > 15) return cudaErrorInvalidValue;
  return dbl ? orth_dispatch<double>(d, k, V, w, H, active, st) : orth_dispatch<float>(d, k, V, w, H, active, st);
}

// ------------------------------------------------------------------ Givens
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }

__global__ void krylov_givens_kernel(KrylovDims d, int k, double2* __restrict__ H, double2* __restrict__ cs,
                                     double2* __restrict__ g, const double* __restrict__ bnorm, int* __restrict__ active,
                                     int* __restrict__ steps, double* __restrict__ est, double rtol, int fixed,
                                     int* nactive) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.S || !active[s]) return;
  double2* Hs = H + (size_t)s * (KMAX + 1) * KMAX;
  double2* css = cs + (size_t)s * KMAX * 2;   // (c as .x, 0) and s complex
  double2* gs = g + (size_t)s * (KMAX + 1);
  // apply previous rotations to column k
  for (int j = 0; j < k; ++j) {
    const double c = css[2 * j].x;
    const double2 sn = css[2 * j + 1];
    const double2 a = Hs[j * KMAX + k], b = Hs[(j + 1) * KMAX + k];
    const double2 na = make_double2(c * a.x + zmul(sn, b).x, c * a.y + zmul(sn, b).y);
    const double2 t = zmul(zconj(sn), a);
    const double2 nb = make_double2(-t.x + c * b.x, -t.y + c * b.y);
    Hs[j * KMAX + k] = na;
    Hs[(j + 1) * KMAX + k] = nb;
  }
  const double2 a = Hs[k * KMAX + k], b = Hs[(k + 1) * KMAX + k];
  const double hk1 = zabs(b);
  const double aa = zabs(a);
  const double r = hypot(aa, hk1);
  double c;
  double2 sn, rr;
  if (r == 0.0) {
    c = 1.0; sn = make_double2(0.0, 0.0); rr = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0; sn = make_double2(1.0, 0.0); rr = b;
  } else {
    const double2 al = make_double2(a.x / aa, a.y / aa);
    c = aa / r;
    const double2 t = zmul(al, zconj(b));
    sn = make_double2(t.x / r, t.y / r);
    rr = make_double2(al.x * r, al.y * r);
  }
  css[2 * k] = make_double2(c, 0.0);
  css[2 * k + 1] = sn;
  Hs[k * KMAX + k] = rr;
  Hs[(k + 1) * KMAX + k] = make_double2(0.0, 0.0);
  const double2 gk = gs[k];
  gs[k] = make_double2(c * gk.x, c * gk.y);
  const double2 t = zmul(zconj(sn), gk);
  gs[k + 1] = make_double2(-t.x, -t.y);
  steps[s] = k + 1;
  const double e = zabs(gs[k + 1]) / (bnorm[s] > 0.0 ? bnorm[s] : 1.0);
  est[s] = e;
  const bool done = (hk1 == 0.0) || (!fixed && e <= rtol);
  if (done) active[s] = 0;
  else atomicAdd(nactive, 1);
}

cudaError_t launch_krylov_givens(KrylovDims d, int k, double2* H, double2* cs, double2* g, const double* bnorm,
                                 int* active, int* steps, double* est, double rtol, int fixed, int* nactive,
                                 cudaStream_t st) {
  krylov_givens_kernel<<<(d.S + 127) / 128, 128, 0, st>>>(d, k, H, cs, g, bnorm, active, steps, est, rtol, fixed,
                                                          nactive);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ solution update
__global__ void krylov_backsolve_kernel(KrylovDims d, const double2* __restrict__ H, const double2* __restrict__ g,
                                        const int* __restrict__ steps, double2* __restrict__ y, int* itot) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.S) return;
  const int k = steps[s];
  itot[s] += k;
  const double2* Hs = H + (size_t)s * (KMAX + 1) * KMAX;
  const double2* gs = g + (size_t)s * (KMAX + 1);
  double2* ys = y + (size_t)s * KMAX;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = gs[i];
    for (int j = i + 1; j < k; ++j) {
      const double2 p = zmul(Hs[i * KMAX + j], ys[j]);
      acc.x -= p.x;
      acc.y -= p.y;
    }
    const double2 dg = Hs[i * KMAX + i];
    const double den = dg.x * dg.x + dg.y * dg.y;
    ys[i] = den > 0.0 ? make_double2((acc.x * dg.x + acc.y * dg.y) / den, (acc.y * dg.x - acc.x * dg.y) / den)
                      : make_double2(0.0, 0.0);
  }
}

template <typename T>
__global__ void __launch_bounds__(KT) krylov_xupdate_kernel(KrylovDims d, const int* __restrict__ steps,
                                                            const double2* __restrict__ y, const cx_t<T>* __restrict__ Z,
                                                            cx_t<T>* __restrict__ x) {
  using C = cx_t<T>;
  const int s = blockIdx.x;
  const int k = steps[s];
  if (k == 0) return;
  const size_t n = d.n, vs = (size_t)d.S * n;
  C yy[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    const double2 v = j < k ? y[(size_t)s * KMAX + j] : make_double2(0.0, 0.0);
    yy[j] = mk<C>((T)v.x, (T)v.y);
  }
  const C* Zs = Z + (size_t)s * n;
  C* xs = x + (size_t)s * n;
  for (size_t i = threadIdx.x; i < n; i += KT) {
    C acc = xs[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) acc = cfma(yy[j], Zs[j * vs + i], acc);
    xs[i] = acc;
  }
}

// complex64 with an even grid: two entries per 16-byte load
__global__ void __launch_bounds__(KT) krylov_xupdate_c64x2_kernel(KrylovDims d, const int* __restrict__ steps,
                                                                  const double2* __restrict__ y,
                                                                  const float4* __restrict__ Z, float4* __restrict__ x) {
  const int s = blockIdx.x;
  const int k = steps[s];
  if (k == 0) return;
  const size_t n2 = d.n / 2, vs2 = (size_t)d.S * n2;
  float2 yy[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    const double2 v = j < k ? y[(size_t)s * KMAX + j] : make_double2(0.0, 0.0);
    yy[j] = make_float2((float)v.x, (float)v.y);
  }
  const float4* Zs = Z + (size_t)s * n2;
  float4* xs = x + (size_t)s * n2;
  for (size_t i = threadIdx.x; i < n2; i += KT) {
    const float4 x0 = xs[i];
    float2 a = make_float2(x0.x, x0.y), b = make_float2(x0.z, x0.w);
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) {
        const float4 z = Zs[j * vs2 + i];
        a = cfma(yy[j], make_float2(z.x, z.y), a);
        b = cfma(yy[j], make_float2(z.z, z.w), b);
      }
    xs[i] = make_float4(a.x, a.y, b.x, b.y);
  }
}

cudaError_t launch_krylov_update(bool dbl, KrylovDims d, const double2* H, const double2* g, const int* steps,
                                 double2* y, const void* Z, void* x, int* itot, cudaStream_t st) {
  krylov_backsolve_kernel<<<(d.S + 127) / 128, 128, 0, st>>>(d, H, g, steps, y, itot);
  if (dbl)
    krylov_xupdate_kernel<double><<<d.S, KT, 0, st>>>(d, steps, y, (const double2*)Z, (double2*)x);
  else if (d.n % 2 == 0 && (uintptr_t)Z % 16 == 0 && (uintptr_t)x % 16 == 0)
    krylov_xupdate_c64x2_kernel<<<d.S, KT, 0, st>>>(d, steps, y, (const float4*)Z, (float4*)x);
  else
    krylov_xupdate_kernel<float><<<d.S, KT, 0, st>>>(d, steps, y, (const float2*)Z, (float2*)x);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ pole combination
template <typename T>
__global__ void pole_combine_kernel(KrylovDims d, int P, const double2* __restrict__ w, double sign, int real_part,
                                    const cx_t<T>* __restrict__ x, cx_t<T>* __restrict__ out) {
  using C = cx_t<T>;
  const size_t total = (size_t)d.N * d.n;   // entry e of pole p's block sits at p * total + e
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    C acc = mk<C>(0, 0);
    for (int p = 0; p < P; ++p) {
      const double2 wp = w[p];
      const C wc = mk<C>((T)(sign * wp.x), (T)(sign * wp.y));
      acc = cfma(wc, x[(size_t)p * total + e], acc);
    }
    if (real_part) acc.y = 0;
    out[e] = acc;
  }
}

// complex64 with an even number of entries: two entries per 16-byte load
__global__ void pole_combine_c64x2_kernel(KrylovDims d, int P, const double2* __restrict__ w, double sign,
                                          int real_part, const float4* __restrict__ x, float4* __restrict__ out) {
  const size_t total2 = (size_t)d.N * d.n / 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total2; e += (size_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f), b = a;
    for (int p = 0; p < P; ++p) {
      const double2 wp = w[p];
      const float2 wc = make_float2((float)(sign * wp.x), (float)(sign * wp.y));
      const float4 v = x[(size_t)p * total2 + e];
      a = cfma(wc, make_float2(v.x, v.y), a);
      b = cfma(wc, make_float2(v.z, v.w), b);
    }
    if (real_part) a.y = b.y = 0.f;
    out[e] = make_float4(a.x, a.y, b.x, b.y);
  }
}

cudaError_t launch_pole_combine(bool dbl, KrylovDims d, int P, const double2* w, double sign, int real_part,
                                const void* x, void* out, cudaStream_t st) {
  const size_t total = (size_t)d.N * d.n;
  const int blocks = (int)((total + 255) / 256 < 4864 ? (total + 255) / 256 : 4864);
  if (dbl)
    pole_combine_kernel<double><<<blocks, 256, 0, st>>>(d, P, w, sign, real_part, (const double2*)x, (double2*)out);
  else if (total % 2 == 0 && (uintptr_t)x % 16 == 0 && (uintptr_t)out % 16 == 0)
    pole_combine_c64x2_kernel<<<blocks, 256, 0, st>>>(d, P, w, sign, real_part, (const float4*)x, (float4*)out);
  else
    pole_combine_kernel<float><<<blocks, 256, 0, st>>>(d, P, w, sign, real_part, (const float2*)x, (float2*)out);
  return cudaGetLastError();
}

__global__ void count_active_kernel(KrylovDims d, const int* __restrict__ active, int* nactive) {
  __shared__ int sh;
  if (threadIdx.x == 0) sh = 0;
  __syncthreads();
  int c = 0;
  for (int s = threadIdx.x; s < d.S; s += blockDim.x) c += active[s] ? 1 : 0;
  atomicAdd(&sh, c);
  __syncthreads();
  if (threadIdx.x == 0) *nactive = sh;
}

cudaError_t launch_count_active(KrylovDims d, const int* active, int* nactive, cudaStream_t st) {
  count_active_kernel<<<1, 1024, 0, st>>>(d, active, nactive);
  return cudaGetLastError();
}

}  // namespace omm
