// Dense block kernels on CUDA cores: Gram products A^H B with a deterministic split-K
// reduction to FP64, tall-skinny block updates (n x N times N x N), axpby, real dot
// products and precision conversion.
//
// Gram (Sec. 2.1 and eq. omm): X^*X, X^*HX and the line-search blocks reduce over the
// grid (length n); partial sums of 32 products are formed in the working precision and
// accumulated in FP64; the split-K partials are summed in a fixed order.
#include "common.cuh"
#include "kernels.h"

#include <map>
#include <mutex>

namespace omm {

cudaError_t raise_smem_limit(const void* func) {
  static std::mutex mu;
  static std::map<const void*, cudaError_t> done;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find(func);
  if (it != done.end()) return it->second;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  done[func] = e;
  return e;
}

namespace {
constexpr int GT = 32;   // Gram tile (outputs per side)
constexpr int GK = 32;   // Gram k-step
constexpr int RED_BLOCKS = 1024;

int gram_splits(int na, int nb, size_t n) {
  const int tiles = ((na + GT - 1) / GT) * ((nb + GT - 1) / GT);
  int ks = (1216 + tiles - 1) / tiles;   // aim at >= 8 CTAs per SM
  const int maxks = (int)((n + 255) / 256);
  if (ks > maxks) ks = maxks;
  if (ks < 1) ks = 1;
  return ks;
}
}  // namespace

size_t gram_work_bytes(int na, int nb, size_t n) {
  return sizeof(double2) * (size_t)gram_splits(na, nb, n) * na * nb;
}

template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const cx_t<T>* __restrict__ A, int na,
                                                           const cx_t<T>* __restrict__ B, int nb, size_t n,
                                                           size_t kchunk, double2* __restrict__ part) {
  using C = cx_t<T>;
  __shared__ C As[GK][GT + 1];
  __shared__ C Bs[GK][GT + 1];
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  const size_t kb = (size_t)blockIdx.z * kchunk;
  const size_t ke = (kb + kchunk < n) ? kb + kchunk : n;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double2 acc64[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc64[a][b] = make_double2(0.0, 0.0);
  for (size_t k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + r * 256;
      const int c = e / GK, kk = e % GK;
      const size_t k = k0 + kk;
      const bool kin = k < ke;
      As[kk][c] = (kin && i0 + c < na) ? A[(size_t)(i0 + c) * n + k] : mk<C>(0, 0);
      Bs[kk][c] = (kin && j0 + c < nb) ? B[(size_t)(j0 + c) * n + k] : mk<C>(0, 0);
    }
    __syncthreads();
    C acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) acc[a][b] = mk<C>(0, 0);
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const C a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const C b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      acc[0][0] = cfmac(a0, b0, acc[0][0]);
      acc[0][1] = cfmac(a0, b1, acc[0][1]);
      acc[1][0] = cfmac(a1, b0, acc[1][0]);
      acc[1][1] = cfmac(a1, b1, acc[1][1]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        acc64[a][b].x += (double)acc[a][b].x;
        acc64[a][b].y += (double)acc[a][b].y;
      }
  }
  double2* out = part + (size_t)blockIdx.z * na * nb;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
      if (i < na && j < nb) out[(size_t)i * nb + j] = acc64[a][b];
    }
}

__global__ void gram_reduce_kernel(const double2* __restrict__ part, int ks, int na, int nb, double2* __restrict__ C,
                                   int ldc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= na * nb) return;
  double2 s = make_double2(0.0, 0.0);
  for (int z = 0; z < ks; ++z) {
    const double2 v = part[(size_t)z * na * nb + idx];
    s.x += v.x;
    s.y += v.y;
  }
  const int i = idx / nb, j = idx % nb;
  C[(size_t)i * ldc + j] = s;
}

cudaError_t launch_gram(bool dbl, const void* A, int na, const void* B, int nb, size_t n, double2* C, int ldc,
                        void* work, cudaStream_t st) {
  if (na <= 0 || nb <= 0) return cudaSuccess;
  const int ks = gram_splits(na, nb, n);
  size_t kchunk = (n + ks - 1) / ks;
  kchunk = (kchunk + GK - 1) / GK * GK;
  dim3 grid((na + GT - 1) / GT, (nb + GT - 1) / GT, ks);
  double2* part = (double2*)work;
  if (dbl)
    gram_partial_kernel<double><<<grid, 256, 0, st>>>((const double2*)A, na, (const double2*)B, nb, n, kchunk, part);
  else
    gram_partial_kernel<float><<<grid, 256, 0, st>>>((const float2*)A, na, (const float2*)B, nb, n, kchunk, part);
  const int tot = na * nb;
  gram_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(part, ks, na, nb, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ block update
// Out[:, j] = a A[:, j] + b B[:, j] + sum_i A[:, i] M1[i][j] + sum_i B[:, i] M2[i][j]
constexpr int BU_R = 64, BU_C = 32, BU_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) block_update_kernel(const cx_t<T>* __restrict__ A, const cx_t<T>* __restrict__ B,
                                                           const cx_t<T>* __restrict__ M1,
                                                           const cx_t<T>* __restrict__ M2, T a, T b, int N, size_t n,
                                                           cx_t<T>* __restrict__ Out) {
  using C = cx_t<T>;
  __shared__ C Xs[BU_K][BU_R];
  __shared__ C Ms[BU_K][BU_C];
  const size_t r0 = (size_t)blockIdx.x * BU_R;
  const int j0 = blockIdx.y * BU_C;
  const int rr = threadIdx.x % BU_R;
  const int jg = (threadIdx.x / BU_R) * 8;   // 0, 8, 16, 24
  const size_t r = r0 + rr;
  C acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = mk<C>(0, 0);
  for (int pass = 0; pass < 2; ++pass) {
    const C* X = pass == 0 ? A : B;
    const C* M = pass == 0 ? M1 : M2;
    for (int i0 = 0; i0 < N; i0 += BU_K) {
      // load X tile: BU_K columns x BU_R rows (1024 elements, 4 per thread)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = threadIdx.x + q * 256;
        const int ii = e / BU_R, ro = e % BU_R;
        const size_t row = r0 + ro;
        Xs[ii][ro] = (i0 + ii < N && row < n) ? X[(size_t)(i0 + ii) * n + row] : mk<C>(0, 0);
      }
      // load M tile: BU_K x BU_C (512 elements, 2 per thread)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int e = threadIdx.x + q * 256;
        const int ii = e / BU_C, jj = e % BU_C;
        Ms[ii][jj] = (i0 + ii < N && j0 + jj < N) ? M[(size_t)(i0 + ii) * N + j0 + jj] : mk<C>(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int ii = 0; ii < BU_K; ++ii) {
        const C x = Xs[ii][rr];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = cfma(x, Ms[ii][jg + q], acc[q]);
      }
      __syncthreads();
    }
  }
  if (r < n) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = j0 + jg + q;
      if (j < N) {
        C v = acc[q];
        if (a != T(0)) { const C x = A[(size_t)j * n + r]; v.x += a * x.x; v.y += a * x.y; }
        if (b != T(0)) { const C y = B[(size_t)j * n + r]; v.x += b * y.x; v.y += b * y.y; }
        Out[(size_t)j * n + r] = v;
      }
    }
  }
}

cudaError_t launch_block_update(bool dbl, const void* A, const void* B, const void* M1, const void* M2, double a,
                                double b, int N, size_t n, void* Out, cudaStream_t st) {
  dim3 grid((unsigned)((n + BU_R - 1) / BU_R), (N + BU_C - 1) / BU_C);
  if (dbl)
    block_update_kernel<double><<<grid, 256, 0, st>>>((const double2*)A, (const double2*)B, (const double2*)M1,
                                                      (const double2*)M2, a, b, N, n, (double2*)Out);
  else
    block_update_kernel<float><<<grid, 256, 0, st>>>((const float2*)A, (const float2*)B, (const float2*)M1,
                                                     (const float2*)M2, (float)a, (float)b, N, n, (float2*)Out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ axpby
template <typename T>
__global__ void axpby_kernel(size_t count, const double2* __restrict__ alpha, const cx_t<T>* __restrict__ X,
                             const double2* __restrict__ beta, cx_t<T>* __restrict__ Y) {
  using C = cx_t<T>;
  const double2 al = alpha ? *alpha : make_double2(1.0, 0.0);
  const double2 be = beta ? *beta : make_double2(0.0, 0.0);
  const C a = mk<C>((T)al.x, (T)al.y), b = mk<C>((T)be.x, (T)be.y);
  const bool usey = beta != nullptr;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    C v = cmul(a, X[i]);
    if (usey) v = cfma(b, Y[i], v);
    Y[i] = v;
  }
}

cudaError_t launch_axpby(bool dbl, size_t count, const double2* alpha, const void* X, const double2* beta, void* Y,
                         cudaStream_t st) {
  const int blocks = (int)((count + 255) / 256 < 4864 ? (count + 255) / 256 : 4864);
  if (count == 0) return cudaSuccess;
  if (dbl)
    axpby_kernel<double><<<blocks, 256, 0, st>>>(count, alpha, (const double2*)X, beta, (double2*)Y);
  else
    axpby_kernel<float><<<blocks, 256, 0, st>>>(count, alpha, (const float2*)X, beta, (float2*)Y);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ real dot
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r += sh[w];
  return r;
}

template <typename T>
__global__ void redot_partial_kernel(size_t count, const cx_t<T>* __restrict__ A, const cx_t<T>* __restrict__ B,
                                     double* __restrict__ part) {
  __shared__ double sh[32];
  T s = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const auto a = A[i];
    const auto b = B[i];
    s += a.x * b.x + a.y * b.y;
  }
  const double r = block_sum((double)s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

__global__ void redot_final_kernel(const double* __restrict__ part, int np, double* res) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  const double r = block_sum(s, sh);
  if (threadIdx.x == 0) *res = r;
}

size_t redot_work_bytes() { return sizeof(double) * RED_BLOCKS; }

cudaError_t launch_redot(bool dbl, size_t count, const void* A, const void* B, double* res, void* work,
                         cudaStream_t st) {
  double* part = (double*)work;
  if (dbl)
    redot_partial_kernel<double><<<RED_BLOCKS, 256, 0, st>>>(count, (const double2*)A, (const double2*)B, part);
  else
    redot_partial_kernel<float><<<RED_BLOCKS, 256, 0, st>>>(count, (const float2*)A, (const float2*)B, part);
  redot_final_kernel<<<1, 1024, 0, st>>>(part, RED_BLOCKS, res);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ convert
template <typename Td, typename Ts>
__global__ void convert_kernel(size_t count, const cx_t<Ts>* __restrict__ s, cx_t<Td>* __restrict__ d) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    d[i] = ccast<cx_t<Td>>(s[i]);
}

cudaError_t launch_convert(bool to_dbl, size_t count, const void* src, void* dst, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)((count + 255) / 256 < 4864 ? (count + 255) / 256 : 4864);
  if (to_dbl)
    convert_kernel<double, float><<<blocks, 256, 0, st>>>(count, (const float2*)src, (double2*)dst);
  else
    convert_kernel<float, double><<<blocks, 256, 0, st>>>(count, (const double2*)src, (float2*)dst);
  return cudaGetLastError();
}

template <typename T>
__global__ void real_part_kernel(size_t count, cx_t<T>* __restrict__ x) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    x[e].y = 0;
}

cudaError_t launch_real_part(bool dbl, size_t count, void* x, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)((count + 255) / 256 < 4864 ? (count + 255) / 256 : 4864);
  if (dbl)
    real_part_kernel<double><<<blocks, 256, 0, st>>>(count, (double2*)x);
  else
    real_part_kernel<float><<<blocks, 256, 0, st>>>(count, (float2*)x);
  return cudaGetLastError();
}

}  // namespace omm

// ------------------------------------------------------------------ Gram without device allocation
// omm_gram_noalloc: the split-K Gram above with its partial sums kept in a fixed device
// array instead of a work buffer, for callers that cannot call cudaMalloc.  The array is
// a file-scope __device__ variable: every GPU that loads the library holds it until the
// process exits, and every call on a device shares it.
#include <mutex>

namespace omm {
namespace {
constexpr size_t kNoAllocPartials = (size_t)1 << 19;   // double2 entries (8 MiB per device)
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocPartials];
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double2* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

}  // namespace omm

extern "C" omm_status omm_gram_noalloc(int precision, const void* A, int na, const void* B, int nb, size_t n, void* C,
                                       void* stream) {
  using namespace omm;
  if ((precision != OMM_FP64 && precision != OMM_MIXED) || !A || !B || !C || na < 1 || nb < 1 || n < 1)
    return OMM_EINVAL;
  if ((size_t)na * nb > kNoAllocPartials) {
    omm_internal_set_cuda_error(cudaErrorInvalidValue, "omm_gram_noalloc: na * nb exceeds the static capacity of 524288 entries",
                                __FILE__, __LINE__);
    return OMM_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    omm_internal_set_cuda_error(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice", __FILE__, __LINE__);
    return OMM_ECUDA;
  }
  double2* part = nullptr;
  {
    // set-up, once per device with that device current: the host-side name of the array
    // is not a device address, so resolve it
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) {
        omm_internal_set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_partials)", __FILE__, __LINE__);
        return OMM_ECUDA;
      }
      g_noalloc_ptr[dev] = (double2*)p;
    }
    part = g_noalloc_ptr[dev];
  }
  // split K so that the partials fit the fixed array (each partial is written before it is read)
  int ks = gram_splits(na, nb, n);
  const int fit = (int)(kNoAllocPartials / ((size_t)na * nb));
  if (ks > fit) ks = fit;
  size_t kchunk = (n + ks - 1) / ks;
  kchunk = (kchunk + GK - 1) / GK * GK;
  ks = (int)((n + kchunk - 1) / kchunk);
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((na + GT - 1) / GT, (nb + GT - 1) / GT, ks);
  if (precision == OMM_FP64)
    gram_partial_kernel<double><<<grid, 256, 0, st>>>((const double2*)A, na, (const double2*)B, nb, n, kchunk, part);
  else
    gram_partial_kernel<float><<<grid, 256, 0, st>>>((const float2*)A, na, (const float2*)B, nb, n, kchunk, part);
  const int tot = na * nb;
  gram_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(part, ks, na, nb, (double2*)C, nb);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    omm_internal_set_cuda_error(e, "omm_gram_noalloc launch", __FILE__, __LINE__);
    return OMM_ECUDA;
  }
  return OMM_OK;
}
