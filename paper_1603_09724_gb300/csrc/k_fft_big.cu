// Multi-pass pseudospectral kernels for grids that do not fit one CTA's shared memory
// (complex double 128^2, 3D 32^3..48^3): one kernel per axis, each CTA transforming a
// tile of lines in shared memory (rows of x, or 16 consecutive x for the y / z lines so
// that global loads stay coalesced).  The last forward axis also applies the k-space
// multiplier (kinetic symbol or Green symbol) and transforms back; the final inverse x
// pass adds (V - s) x for the H-apply.
//
//   H-apply  Y = F^-1 (T(k) F x) + (V - s_g) x     (Sec. 4 eq. ex1mat)
//   Green    Out = F^-1 (Ghat_g(k) F b)            (Sec. 3.2 eq. GLu); the Q stencil is a
//            separate gather kernel (stencil_kernel)
#include "fft.cuh"
#include "kernels.h"

namespace omm {

namespace {

constexpr int BT = 256;   // threads
constexpr int TX = 16;    // x columns per tile for y / z lines
constexpr int RX = 16;    // rows per tile for x lines

template <int M> struct RowTile {   // RX lines along x, pitch M + 1
  static constexpr int NL = RX;
  static constexpr int ESTR = 1;
  static constexpr int Mv = M;
  __device__ __forceinline__ static int base(int l) { return l * (M + 1); }
};
template <int M> struct ColTile {   // TX lines, element stride TX + 1
  static constexpr int NL = TX;
  static constexpr int ESTR = TX + 1;
  static constexpr int Mv = M;
  __device__ __forceinline__ static int base(int l) { return l; }
};

// adapter: fft::pass expects LN::M
template <class TL> struct LN_ : TL { static constexpr int M = TL::Mv; };

template <int SGN, class LN, typename C> __device__ __forceinline__ void axis_tile(C* s, const C* tw) {
  fft::axis<SGN, LN_<LN>, BT>(s, tw);
}

}  // namespace

// ---- x pass: RX rows per CTA.  mode 0: forward, in -> out.  mode 1: inverse and finish
// the H-apply: out = F_x^-1 in + (V - s) X (the 1/n is folded into the multiplier).
// mode 2: inverse only.  in and out may alias (each CTA reads its tile before writing).
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(BT) xpass_kernel(const cx_t<T>* in, cx_t<T>* out,
                                                   size_t n, const cx_t<T>* __restrict__ tw, const T* __restrict__ V,
                                                   const cx_t<T>* __restrict__ X, const double2* __restrict__ shifts,
                                                   int cpg, const int* __restrict__ active, int tiles_per_col) {
  using C = cx_t<T>;
  __shared__ C s[RX * (M + 1)];
  __shared__ C t[M];
  const int col = blockIdx.x / tiles_per_col, tile = blockIdx.x % tiles_per_col;
  if (active && !active[col]) return;
  const size_t base = (size_t)col * n + (size_t)tile * RX * M;
  for (int i = threadIdx.x; i < M; i += BT) t[i] = tw[i];
  for (int i = threadIdx.x; i < RX * M; i += BT) s[(i / M) * (M + 1) + i % M] = in[base + i];
  __syncthreads();
  if (MODE == 0) axis_tile<-1, RowTile<M>>(s, t);
  else axis_tile<+1, RowTile<M>>(s, t);
  if (MODE != 1) {
    for (int i = threadIdx.x; i < RX * M; i += BT) out[base + i] = s[(i / M) * (M + 1) + i % M];
  } else {
    const double2 sh = shifts[col / cpg];
    const T sr = (T)sh.x, si = (T)sh.y;
    const size_t off = (size_t)tile * RX * M;
    for (int i = threadIdx.x; i < RX * M; i += BT) {
      const C xi = X[base + i];
      const T vr = V[off + i] - sr;
      C r = s[(i / M) * (M + 1) + i % M];
      r.x += vr * xi.x + si * xi.y;
      r.y += vr * xi.y - si * xi.x;
      out[base + i] = r;
    }
  }
}

// ---- y or z pass over TX consecutive x columns.  STRIDE = M (y) or M*M (z).
// mode 0: forward; 1: inverse; 2: forward, multiply, inverse (kinetic, 1/n folded);
// 3: forward, multiply by the Green table of the column's group, inverse.
template <typename T, int M, int DIM, int AX, int MODE>
__global__ void __launch_bounds__(BT) lpass_kernel(cx_t<T>* __restrict__ buf, size_t n, const cx_t<T>* __restrict__ tw,
                                                   double kin_over_n, const cx_t<T>* __restrict__ ghat, int cpg,
                                                   const int* __restrict__ active, int tiles_per_col) {
  using C = cx_t<T>;
  __shared__ C s[M * (TX + 1)];
  __shared__ C t[M];
  const int col = blockIdx.x / tiles_per_col, tile = blockIdx.x % tiles_per_col;
  if (active && !active[col]) return;
  constexpr int XT = M / TX;                // x tiles per line of the other axis
  const int x0 = (tile % XT) * TX;
  const int other = tile / XT;              // y (for z lines) or z (for y lines)
  constexpr size_t STRIDE = (AX == 1) ? (size_t)M : (size_t)M * M;
  const size_t obase = (AX == 1) ? (size_t)other * M * M : (size_t)other * M;
  C* g = buf + (size_t)col * n;
  for (int i = threadIdx.x; i < M; i += BT) t[i] = tw[i];
  for (int i = threadIdx.x; i < M * TX; i += BT) {
    const int e = i / TX, xx = i % TX;
    s[e * (TX + 1) + xx] = g[obase + (size_t)e * STRIDE + x0 + xx];
  }
  __syncthreads();
  if (MODE == 1) {
    axis_tile<+1, ColTile<M>>(s, t);
  } else {
    axis_tile<-1, ColTile<M>>(s, t);
    if (MODE >= 2) {
      const C* gh = (MODE == 3) ? ghat + (size_t)(col / cpg) * n : nullptr;
      for (int i = threadIdx.x; i < M * TX; i += BT) {
        const int e = i / TX, xx = i % TX;
        const size_t flat = obase + (size_t)e * STRIDE + x0 + xx;
        C& v = s[e * (TX + 1) + xx];
        if (MODE == 2) {
          const int ix = (int)(flat % M), iy = (int)((flat / M) % M), iz = (DIM == 3) ? (int)(flat / ((size_t)M * M)) : 0;
          const int kx = fft::signed_k(ix, M), ky = fft::signed_k(iy, M), kz = (DIM == 3) ? fft::signed_k(iz, M) : 0;
          v = cscale(v, (T)(kin_over_n * (double)(kx * kx + ky * ky + kz * kz)));
        } else {
          v = cmul(v, gh[flat]);
        }
      }
      __syncthreads();
      axis_tile<+1, ColTile<M>>(s, t);
    }
  }
  for (int i = threadIdx.x; i < M * TX; i += BT) {
    const int e = i / TX, xx = i % TX;
    g[obase + (size_t)e * STRIDE + x0 + xx] = s[e * (TX + 1) + xx];
  }
}

// ---- xy slab pass (3D): one CTA transforms a whole z-slab (M x M) along x and y in shared
// memory, so a 3D transform is two kernels (xy slabs, z pencils) instead of three.
// mode 0: forward, in -> out.  mode 1: inverse and finish the H-apply:
// out = F_xy^-1 in + (V - s) X.  mode 2: inverse only.  in and out may alias.
template <typename T, int M>
struct SlabCfg {
  using LY = fft::Layout<M, M, 1>;
  static constexpr size_t smem = sizeof(cx_t<T>) * (LY::SIZE + M);
};

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(BT) xyslab_kernel(const cx_t<T>* in, cx_t<T>* out, size_t n,
                                                    const cx_t<T>* __restrict__ tw, const T* __restrict__ V,
                                                    const cx_t<T>* __restrict__ X, const double2* __restrict__ shifts,
                                                    int cpg, const int* __restrict__ active) {
  using C = cx_t<T>;
  using LY = typename SlabCfg<T, M>::LY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  C* t = s + LY::SIZE;
  const int col = blockIdx.x / M, z = blockIdx.x % M;
  if (active && !active[col]) return;
  const size_t base = (size_t)col * n + (size_t)z * M * M;
  for (int i = threadIdx.x; i < M; i += BT) t[i] = tw[i];
  for (int i = threadIdx.x; i < M * M; i += BT) s[LY::at_flat(i)] = in[base + i];
  __syncthreads();
  if (MODE == 0) fft::transform<-1, LY, 1, BT>(s, t, t, t);
  else fft::transform<+1, LY, 1, BT>(s, t, t, t);
  if (MODE != 1) {
    for (int i = threadIdx.x; i < M * M; i += BT) out[base + i] = s[LY::at_flat(i)];
  } else {
    const double2 sh = shifts[col / cpg];
    const T sr = (T)sh.x, si = (T)sh.y;
    const size_t off = (size_t)z * M * M;
    for (int i = threadIdx.x; i < M * M; i += BT) {
      const C xi = X[base + i];
      const T vr = V[off + i] - sr;
      C r = s[LY::at_flat(i)];
      r.x += vr * xi.x + si * xi.y;
      r.y += vr * xi.y - si * xi.x;
      out[base + i] = r;
    }
  }
}

// slabs up to this many bytes of shared memory take the two-kernel 3D path
constexpr size_t kSlabSmemMax = 100 * 1024;

template <typename T, int M>
static bool slab_ok(int dim) {
  return dim == 3 && SlabCfg<T, M>::smem <= kSlabSmemMax;
}

template <typename T, int M, int MODE>
static cudaError_t launch_xyslab(const cx_t<T>* in, cx_t<T>* out, size_t n, int ncols, const cx_t<T>* tw,
                                 const T* V, const cx_t<T>* X, const double2* shifts, int cpg, const int* active,
                                 cudaStream_t st) {
  auto k = xyslab_kernel<T, M, MODE>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  k<<<ncols * M, BT, SlabCfg<T, M>::smem, st>>>(in, out, n, tw, V, X, shifts, cpg, active);
  return cudaGetLastError();
}

// ---- Q stencil on a natural-order grid function: out[j] = sum_t q_t in[j + o_t], stored at
// out[iperm[j]] when a permutation is given
template <typename T>
__global__ void stencil_kernel(const cx_t<T>* __restrict__ in, cx_t<T>* __restrict__ out, int dim, int m, size_t n,
                               const cx_t<T>* __restrict__ q, int nq, int cpg, const int* __restrict__ active,
                               const int* __restrict__ iperm) {
  using C = cx_t<T>;
  const int col = blockIdx.y;
  if (active && !active[col]) return;
  const C* qs = q + (size_t)(col / cpg) * nq;
  const C* g = in + (size_t)col * n;
  const int r = (nq == 1) ? 0 : 1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % m), iy = (int)((i / m) % m), iz = (dim == 3) ? (int)(i / ((size_t)m * m)) : 0;
    C acc = mk<C>(0, 0);
    int qi = 0;
    const int rz = (dim == 3) ? r : 0;
    for (int dz = -rz; dz <= rz; ++dz)
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx, ++qi) {
          const int xx = (ix + dx + m) % m, yy = (iy + dy + m) % m, zz = (dim == 3) ? (iz + dz + m) % m : 0;
          acc = cfma(qs[qi], g[xx + (size_t)m * (yy + (size_t)m * zz)], acc);
        }
    out[(size_t)col * n + (iperm ? (size_t)iperm[i] : i)] = acc;
  }
}

// ------------------------------------------------------------------ drivers
template <typename T, int M>
static cudaError_t happly_big_t(int dim, const void* X, void* Y, int ncols, const void* V, const double2* shifts,
                                int cpg, const void* tw, double kin_over_n, const int* active, void* tmp,
                                cudaStream_t st) {
  using C = cx_t<T>;
  const size_t n = (dim == 3) ? (size_t)M * M * M : (size_t)M * M;
  const int xt = (int)(n / M / RX);
  const int lt = (dim == 3) ? (M / TX) * M : (M / TX);
  const C* x = (const C*)X;
  C* w = (C*)tmp;
  const C* t = (const C*)tw;
  if (slab_ok<T, M>(dim)) {   // xy slabs forward, z pencils forward-multiply-inverse, xy slabs inverse + V
    cudaError_t e = launch_xyslab<T, M, 0>(x, w, n, ncols, t, nullptr, nullptr, nullptr, 1, active, st);
    if (e != cudaSuccess) return e;
    lpass_kernel<T, M, 3, 2, 2><<<ncols * lt, BT, 0, st>>>(w, n, t, kin_over_n, nullptr, 1, active, lt);
    return launch_xyslab<T, M, 1>(w, (C*)Y, n, ncols, t, (const T*)V, x, shifts, cpg, active, st);
  }
  xpass_kernel<T, M, 0><<<ncols * xt, BT, 0, st>>>(x, w, n, t, nullptr, nullptr, nullptr, 1, active, xt);
  if (dim == 2) {
    lpass_kernel<T, M, 2, 1, 2><<<ncols * lt, BT, 0, st>>>(w, n, t, kin_over_n, nullptr, 1, active, lt);
  } else {
    lpass_kernel<T, M, 3, 1, 0><<<ncols * lt, BT, 0, st>>>(w, n, t, kin_over_n, nullptr, 1, active, lt);
    lpass_kernel<T, M, 3, 2, 2><<<ncols * lt, BT, 0, st>>>(w, n, t, kin_over_n, nullptr, 1, active, lt);
    lpass_kernel<T, M, 3, 1, 1><<<ncols * lt, BT, 0, st>>>(w, n, t, kin_over_n, nullptr, 1, active, lt);
  }
  xpass_kernel<T, M, 1><<<ncols * xt, BT, 0, st>>>(w, (C*)Y, n, t, (const T*)V, x, shifts, cpg, active, xt);
  return cudaGetLastError();
}

template <typename T, int M>
static cudaError_t greenq_big_t(int dim, const void* B, void* Out, int ncols, const void* ghat, const void* q, int nq,
                                int cpg, const void* tw, const int* active, const int* iperm, void* tmp,
                                cudaStream_t st) {
  using C = cx_t<T>;
  const size_t n = (dim == 3) ? (size_t)M * M * M : (size_t)M * M;
  const int xt = (int)(n / M / RX);
  const int lt = (dim == 3) ? (M / TX) * M : (M / TX);
  C* w = (C*)tmp;
  const C* t = (const C*)tw;
  const C* gh = (const C*)ghat;
  const int sb = (int)((n + 255) / 256 < 256 ? (n + 255) / 256 : 256);
  if (slab_ok<T, M>(dim)) {
    cudaError_t e = launch_xyslab<T, M, 0>((const C*)B, w, n, ncols, t, nullptr, nullptr, nullptr, 1, active, st);
    if (e != cudaSuccess) return e;
    lpass_kernel<T, M, 3, 2, 3><<<ncols * lt, BT, 0, st>>>(w, n, t, 0.0, gh, cpg, active, lt);
    e = launch_xyslab<T, M, 2>(w, w, n, ncols, t, nullptr, nullptr, nullptr, 1, active, st);
    if (e != cudaSuccess) return e;
    stencil_kernel<T><<<dim3(sb, ncols), 256, 0, st>>>(w, (C*)Out, dim, M, n, (const C*)q, nq, cpg, active, iperm);
    return cudaGetLastError();
  }
  xpass_kernel<T, M, 0><<<ncols * xt, BT, 0, st>>>((const C*)B, w, n, t, nullptr, nullptr, nullptr, 1, active, xt);
  if (dim == 2) {
    lpass_kernel<T, M, 2, 1, 3><<<ncols * lt, BT, 0, st>>>(w, n, t, 0.0, gh, cpg, active, lt);
  } else {
    lpass_kernel<T, M, 3, 1, 0><<<ncols * lt, BT, 0, st>>>(w, n, t, 0.0, gh, cpg, active, lt);
    lpass_kernel<T, M, 3, 2, 3><<<ncols * lt, BT, 0, st>>>(w, n, t, 0.0, gh, cpg, active, lt);
    lpass_kernel<T, M, 3, 1, 1><<<ncols * lt, BT, 0, st>>>(w, n, t, 0.0, gh, cpg, active, lt);
  }
  xpass_kernel<T, M, 2><<<ncols * xt, BT, 0, st>>>(w, w, n, t, nullptr, nullptr, nullptr, 1, active, xt);
  stencil_kernel<T><<<dim3(sb, ncols), 256, 0, st>>>(w, (C*)Out, dim, M, n, (const C*)q, nq, cpg, active, iperm);
  return cudaGetLastError();
}

// kernels one call launches (for the launch counts of the profiler)
int big_fft_launches(int dim, int m, bool dbl, bool greenq) {
  size_t smem = (dbl ? sizeof(double2) : sizeof(float2)) * ((size_t)(m + 1) * m + m);
  const bool slab = dim == 3 && smem <= kSlabSmemMax;
  if (slab) return greenq ? 4 : 3;
  return (dim == 3 ? 5 : 3) + (greenq ? 1 : 0);
}

bool big_fft_supported(int dim, int m) {
  if (m % TX != 0) return false;
  switch (m) {
    case 16: case 32: case 48: case 64: case 96: case 128: return dim == 2 || dim == 3;
    default: return false;
  }
}

cudaError_t launch_happly_big(bool dbl, int dim, int m, const void* X, void* Y, int ncols, const void* V,
                              const double2* shifts, int cpg, const void* tw, double kin_over_n, const int* active,
                              void* tmp, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
#define C_(M)                                                                                                  \
  case M:                                                                                                      \
    return dbl ? happly_big_t<double, M>(dim, X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, tmp, st)   \
               : happly_big_t<float, M>(dim, X, Y, ncols, V, shifts, cpg, tw, kin_over_n, active, tmp, st);
  switch (m) {
    C_(16) C_(32) C_(48) C_(64) C_(96) C_(128)
    default: break;
  }
#undef C_
  return cudaErrorInvalidValue;
}

cudaError_t launch_greenq_big(bool dbl, int dim, int m, const void* B, void* Out, int ncols, const void* ghat,
                              const void* q, int nq, int cpg, const void* tw, const int* active, const int* iperm,
                              void* tmp, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
#define C_(M)                                                                                              \
  case M:                                                                                                  \
    return dbl ? greenq_big_t<double, M>(dim, B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, tmp, st)       \
               : greenq_big_t<float, M>(dim, B, Out, ncols, ghat, q, nq, cpg, tw, active, iperm, tmp, st);
  switch (m) {
    C_(16) C_(32) C_(48) C_(64) C_(96) C_(128)
    default: break;
  }
#undef C_
  return cudaErrorInvalidValue;
}

}  // namespace omm
