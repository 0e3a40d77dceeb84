// Fused pseudospectral kernels: one CTA per grid function, whole grid in shared memory.
//
//  happly : Y = F^-1 (T(k) F x) + (V - s_g) x     (Sec. 4 eq. ex1mat; shifted for eq. lst)
//  greenq : out = Q (F^-1 (Ghat_g(k) F b))          (Sec. 3.2 eqs. GLu / QG: Q (G b))
//           optionally stored through a permutation (out[iperm[i]]), e.g. straight into the
//           nested-dissection order of the triangular solves that consume it
//
// s_g / Ghat_g / q_g depend on the column group g = col / cols_per_group (one group per
// pole when the columns of all P shifted systems are batched).  T(k) = c |k|^2 with the
// signed wave numbers k in [-m/2, m/2).
#include "fft.cuh"
#include "kernels.h"

namespace omm {

template <typename T, int M, int D>
struct GridCfg {
  static constexpr int MX = M, MY = M, MZ = (D == 3 ? M : 1);
  using LY = fft::Layout<MX, MY, MZ>;
  static constexpr int N = MX * MY * MZ;
  static constexpr int NT = (N >= 8192) ? 512 : 256;
  static constexpr size_t smem = sizeof(cx_t<T>) * (LY::SIZE + M);
};

// Point-wise multipliers applied as the first pass of the inverse transform loads its
// inputs (fft::transform's pre; that pass runs along y in 2D, z in 3D): the grid point of
// input (line l, position pos) is x = l % M and y = pos (2D), or y = l / M and z = pos (3D).
template <int M, int D>
__device__ __forceinline__ int flat_of_inverse_line(int l, int pos) {
  return D == 3 ? pos * M * M + l : pos * M + l;
}

// the kinetic symbol c |k|^2 (the H-apply)
template <typename T, int M, int D>
struct KineticPre {
  T kc;
  __device__ __forceinline__ cx_t<T> operator()(cx_t<T> v, int l, int pos) const {
    const int kx = fft::signed_k(l % M, M);
    const int ky = fft::signed_k(D == 3 ? l / M : pos, M);
    const int kz = D == 3 ? fft::signed_k(pos, M) : 0;
    return cscale(v, kc * (T)(kx * kx + ky * ky + kz * kz));
  }
};

// the Green symbol of the column's group (the Green kernel)
template <typename T, int M, int D>
struct GreenPre {
  const cx_t<T>* gh;
  __device__ __forceinline__ cx_t<T> operator()(cx_t<T> v, int l, int pos) const {
    return cmul(v, gh[flat_of_inverse_line<M, D>(l, pos)]);
  }
};

// The grid function x into the padded shared-memory layout with cp.async (global to shared
// memory without a register round trip, every copy of the thread in flight at once); the
// caller's __syncthreads follows.
template <typename T, int M, int D>
__device__ __forceinline__ void load_grid_async(cx_t<T>* s, const cx_t<T>* __restrict__ x) {
  using G = GridCfg<T, M, D>;
  using LY = typename G::LY;
  for (int i = threadIdx.x; i < G::N; i += G::NT) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s + LY::at_flat(i));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(x + i), "n"(sizeof(cx_t<T>)) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename T, int M, int D>
__global__ void __launch_bounds__(GridCfg<T, M, D>::NT)
happly_kernel(const cx_t<T>* __restrict__ X, cx_t<T>* __restrict__ Y, const T* __restrict__ V,
              const double2* __restrict__ shifts, int cols_per_group, const cx_t<T>* __restrict__ tw,
              double kin_over_n, const int* __restrict__ active) {
  using C = cx_t<T>;
  using G = GridCfg<T, M, D>;
  using LY = typename G::LY;
  constexpr int NT = G::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  C* t = s + LY::SIZE;
  const int col = blockIdx.x;
  if (active && !active[col]) return;
  const C* x = X + (size_t)col * G::N;
  for (int i = threadIdx.x; i < M; i += NT) t[i] = tw[i];
  // (plain loads: with cp.async the H-apply measured slower, its epilogue re-reads x)
  for (int i = threadIdx.x; i < G::N; i += NT) s[LY::at_flat(i)] = x[i];
  __syncthreads();
  fft::transform<-1, LY, G::MZ, NT>(s, t, t, t);
  fft::transform<+1, LY, G::MZ, NT>(s, t, t, t, KineticPre<T, M, D>{(T)kin_over_n});
  const double2 sh = shifts[col / cols_per_group];
  const T sr = (T)sh.x, si = (T)sh.y;
  C* y = Y + (size_t)col * G::N;
  for (int i = threadIdx.x; i < G::N; i += NT) {
    const C xi = x[i];
    const T vr = V[i] - sr;
    // (V - s) x = (vr - i si) x
    C r = s[LY::at_flat(i)];
    r.x += vr * xi.x + si * xi.y;
    r.y += vr * xi.y - si * xi.x;
    y[i] = r;
  }
}

template <typename T, int M, int D>
__global__ void __launch_bounds__(GridCfg<T, M, D>::NT)
greenq_kernel(const cx_t<T>* __restrict__ B, cx_t<T>* __restrict__ Out, const cx_t<T>* __restrict__ ghat,
              const cx_t<T>* __restrict__ q, int nq, int cols_per_group, const cx_t<T>* __restrict__ tw,
              const int* __restrict__ active, const int* __restrict__ iperm) {
  using C = cx_t<T>;
  using G = GridCfg<T, M, D>;
  using LY = typename G::LY;
  constexpr int NT = G::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  C* t = s + LY::SIZE;
  __shared__ C qs[27];
  const int col = blockIdx.x;
  if (active && !active[col]) return;
  const int g = col / cols_per_group;
  const C* b = B + (size_t)col * G::N;
  for (int i = threadIdx.x; i < M; i += NT) t[i] = tw[i];
  for (int i = threadIdx.x; i < nq; i += NT) qs[i] = q[(size_t)g * nq + i];
  load_grid_async<T, M, D>(s, b);
  __syncthreads();
  fft::transform<-1, LY, G::MZ, NT>(s, t, t, t);
  fft::transform<+1, LY, G::MZ, NT>(s, t, t, t, GreenPre<T, M, D>{ghat + (size_t)g * G::N});
  C* o = Out + (size_t)col * G::N;
  if constexpr (D == 2 && NT % M == 0 && M % (NT / M) == 0) {
    if (nq == 9) {
      // the 3 x 3 box in 2D: each thread walks a strip of RPS consecutive rows of one grid
      // column with the three rows around the current one in registers, so each output
      // reads three new values (same terms, same order as the loop below)
      constexpr int RPS = M / (NT / M);
      const int ix = threadIdx.x % M, y0 = (threadIdx.x / M) * RPS;
      const int xm = (ix + M - 1) % M, xp = (ix + 1) % M;
      C w[3][3];
      auto row = [&](int yy, C* v) {
        v[0] = s[LY::at(xm, yy, 0)];
        v[1] = s[LY::at(ix, yy, 0)];
        v[2] = s[LY::at(xp, yy, 0)];
      };
      row((y0 + M - 1) % M, w[0]);
      row(y0, w[1]);
#pragma unroll 4
      for (int rr = 0; rr < RPS; ++rr) {
        const int y = y0 + rr;
        row((y + 1) % M, w[2]);
        C acc = mk<C>(0, 0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) acc = cfma(qs[dy * 3 + dx], w[dy][dx], acc);
        const int i = y * M + ix;
        o[iperm ? iperm[i] : i] = acc;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          w[0][dx] = w[1][dx];
          w[1][dx] = w[2][dx];
        }
      }
      return;
    }
  }
  const int r = (nq == 1) ? 0 : 1;   // delta stencil (kinetic inverse only) or the 3^d box
  for (int i = threadIdx.x; i < G::N; i += NT) {
    const int ix = i % M, iy = (i / M) % M, iz = i / (M * M);
    C acc = mk<C>(0, 0);
    int qi = 0;
    const int dzr = (D == 3) ? r : 0;
    for (int dz = -dzr; dz <= dzr; ++dz)
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx, ++qi) {
          const int xx = (ix + dx + M) % M, yy = (iy + dy + M) % M, zz = (D == 3) ? (iz + dz + M) % M : 0;
          acc = cfma(qs[qi], s[LY::at(xx, yy, zz)], acc);
        }
    o[iperm ? iperm[i] : i] = acc;
  }
}

// ---------------------------------------------------------------- dispatch
template <typename T, int M, int D>
static cudaError_t launch_happly_t(const void* X, void* Y, int ncols, const void* V, const double2* shifts,
                                   int cpg, const void* tw, double kin_over_n, const int* active, cudaStream_t st) {
  using G = GridCfg<T, M, D>;
  auto k = happly_kernel<T, M, D>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  k<<<ncols, G::NT, G::smem, st>>>((const cx_t<T>*)X, (cx_t<T>*)Y, (const T*)V, shifts, cpg,
                                   (const cx_t<T>*)tw, kin_over_n, active);
  return cudaGetLastError();
}

template <typename T, int M, int D>
static cudaError_t launch_greenq_t(const void* B, void* Out, int ncols, const void* ghat, const void* q, int nq,
                                   int cpg, const void* tw, const int* active, const int* iperm, cudaStream_t st) {
  using G = GridCfg<T, M, D>;
  auto k = greenq_kernel<T, M, D>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  k<<<ncols, G::NT, G::smem, st>>>((const cx_t<T>*)B, (cx_t<T>*)Out, (const cx_t<T>*)ghat, (const cx_t<T>*)q, nq,
                                   cpg, (const cx_t<T>*)tw, active, iperm);
  return cudaGetLastError();
}

#define OMM_GRID_CASES_2D(X_) X_(8) X_(12) X_(16) X_(24) X_(32) X_(36) X_(48) X_(64) X_(72) X_(96)
#define OMM_GRID_CASES_3D(X_) X_(4) X_(6) X_(8) X_(12) X_(16)

bool fused_fft_supported(int dim, int m, bool dbl) {
  if (dim == 2) {
    switch (m) {
#define C_(M) case M: return true;
      OMM_GRID_CASES_2D(C_)
#undef C_
      case 128: return !dbl;
      default: return false;
    }
  }
  if (dim == 3) {
    switch (m) {
#define C_(M) case M: return true;
      OMM_GRID_CASES_3D(C_)
#undef C_
      default: return false;
    }
  }
  return false;
}

cudaError_t launch_happly(bool dbl, int dim, int m, const void* X, void* Y, int ncols, const void* V,
                          const double2* shifts, int cpg, const void* tw, double kin_over_n, const int* active,
                          cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
#define C2_(M)                                                                                        \
  case M:                                                                                             \
    return dbl ? launch_happly_t<double, M, 2>(X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, st)      \
               : launch_happly_t<float, M, 2>(X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, st);
#define C3_(M)                                                                                        \
  case M:                                                                                             \
    return dbl ? launch_happly_t<double, M, 3>(X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, st)      \
               : launch_happly_t<float, M, 3>(X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, st);
  if (dim == 2) {
    switch (m) {
      OMM_GRID_CASES_2D(C2_)
      case 128:
        if (!dbl) return launch_happly_t<float, 128, 2>(X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, st);
        break;
      default: break;
    }
  } else if (dim == 3) {
    switch (m) { OMM_GRID_CASES_3D(C3_) default: break; }
  }
#undef C2_
#undef C3_
  return cudaErrorInvalidValue;
}

cudaError_t launch_greenq(bool dbl, int dim, int m, const void* B, void* Out, int ncols, const void* ghat,
                          const void* q, int nq, int cpg, const void* tw, const int* active, const int* iperm,
                          cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
#define C2_(M)                                                                                        \
  case M:                                                                                             \
    return dbl ? launch_greenq_t<double, M, 2>(B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, st)              \
               : launch_greenq_t<float, M, 2>(B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, st);
#define C3_(M)                                                                                        \
  case M:                                                                                             \
    return dbl ? launch_greenq_t<double, M, 3>(B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, st)              \
               : launch_greenq_t<float, M, 3>(B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, st);
  if (dim == 2) {
    switch (m) {
      OMM_GRID_CASES_2D(C2_)
      case 128:
        if (!dbl) return launch_greenq_t<float, 128, 2>(B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, st);
        break;
      default: break;
    }
  } else if (dim == 3) {
    switch (m) { OMM_GRID_CASES_3D(C3_) default: break; }
  }
#undef C2_
#undef C3_
  return cudaErrorInvalidValue;
}

}  // namespace omm
