// Shared-memory-resident mixed-radix FFT for one periodic grid function per CTA.
//
// The whole grid (2D up to 128^2 in complex float, 96^2 in complex double; small 3D
// grids) lives in shared memory with the x rows padded by one element, so that a warp
// whose lanes take consecutive lines (rows or columns) touches consecutive banks.  Each
// axis transform is a sequence of in-place Stockham (self-sorting) passes: every thread
// loads its butterflies' R inputs into registers, applies the twiddles, does a radix-R
// DFT, and after a barrier stores the R outputs at their sorted positions.  Radices
// 2, 3, 4, 8, 16 cover the grid sizes 2^a 3^b used here.  Twiddles e^{-2 pi i k/M}
// come from a table computed on the host in double precision with libm.
#pragma once
#include "common.cuh"

namespace omm {
namespace fft {

// ---------------------------------------------------------------- radix kernels
// In-place y_k = sum_r a_r w^{rk}, w = exp(SGN * 2 pi i / R).

template <int SGN, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
  C t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <int SGN, typename C> __device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  using T = decltype(a0.x);
  const T h = T(0.8660254037844386467637231707529362);  // sqrt(3)/2
  C s = cadd(a1, a2), d = csub(a1, a2);
  C m = mk<C>(a0.x - T(0.5) * s.x, a0.y - T(0.5) * s.y);
  C r = cscale(cmuli<SGN>(d), h);
  a0 = cadd(a0, s);
  a1 = cadd(m, r);
  a2 = csub(m, r);
}

template <int SGN, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmuli<SGN>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int SGN, typename C> __device__ __forceinline__ void dft8(C* a) {
  using T = decltype(a[0].x);
  const T c = T(0.7071067811865475244008443621048490);  // sqrt(1/2)
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<SGN>(e0, e1, e2, e3);
  dft4<SGN>(o0, o1, o2, o3);
  o1 = cmul(o1, mk<C>(c, SGN * c));
  o2 = cmuli<SGN>(o2);
  o3 = cmul(o3, mk<C>(-c, SGN * c));
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <int SGN, typename C> __device__ __forceinline__ void dft16(C* a) {
  using T = decltype(a[0].x);
  // cos(pi k / 8), sin(pi k / 8), k = 0..7
  const T cs[8] = {T(1.0), T(0.9238795325112867561281831893967883), T(0.7071067811865475244008443621048490),
                   T(0.3826834323650897717284599840303989), T(0.0), T(-0.3826834323650897717284599840303989),
                   T(-0.7071067811865475244008443621048490), T(-0.9238795325112867561281831893967883)};
  const T sn[8] = {T(0.0), T(0.3826834323650897717284599840303989), T(0.7071067811865475244008443621048490),
                   T(0.9238795325112867561281831893967883), T(1.0), T(0.9238795325112867561281831893967883),
                   T(0.7071067811865475244008443621048490), T(0.3826834323650897717284599840303989)};
  C e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
  dft8<SGN>(e);
  dft8<SGN>(o);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    C t = (k == 0) ? o[k] : cmul(o[k], mk<C>(cs[k], SGN * sn[k]));
    a[k] = cadd(e[k], t);
    a[k + 8] = csub(e[k], t);
  }
}

template <int R, int SGN, typename C> __device__ __forceinline__ void dft(C* a) {
  if constexpr (R == 2) dft2<SGN>(a[0], a[1]);
  else if constexpr (R == 3) dft3<SGN>(a[0], a[1], a[2]);
  else if constexpr (R == 4) dft4<SGN>(a[0], a[1], a[2], a[3]);
  else if constexpr (R == 8) dft8<SGN>(a);
  else if constexpr (R == 16) dft16<SGN>(a);
  else static_assert(R == 2, "unsupported radix");
}

// ---------------------------------------------------------------- plans
// Radix sequence per transform length (Stockham order: first pass has NS = 1).
template <int M> struct Plan;
#define OMM_PLAN(M, NP, A, B, C_, D) \
  template <> struct Plan<M> { static constexpr int np = NP, r0 = A, r1 = B, r2 = C_, r3 = D; };
OMM_PLAN(4, 1, 4, 1, 1, 1)
OMM_PLAN(6, 2, 2, 3, 1, 1)
OMM_PLAN(8, 1, 8, 1, 1, 1)
OMM_PLAN(12, 2, 4, 3, 1, 1)
OMM_PLAN(16, 1, 16, 1, 1, 1)
OMM_PLAN(24, 2, 8, 3, 1, 1)
OMM_PLAN(32, 2, 8, 4, 1, 1)
OMM_PLAN(36, 3, 4, 3, 3, 1)
OMM_PLAN(48, 2, 16, 3, 1, 1)
OMM_PLAN(64, 2, 16, 4, 1, 1)
OMM_PLAN(72, 3, 8, 3, 3, 1)
OMM_PLAN(96, 3, 16, 2, 3, 1)
OMM_PLAN(108, 4, 4, 3, 3, 3)
OMM_PLAN(128, 2, 16, 8, 1, 1)
#undef OMM_PLAN

// ---------------------------------------------------------------- layout
// Grid (x fastest) in shared memory with rows padded to PX = MX + 1 elements.
template <int MX, int MY, int MZ> struct Layout {
  static constexpr int PX = MX + 1;
  static constexpr int N = MX * MY * MZ;
  static constexpr int SIZE = PX * MY * MZ;
  __device__ __forceinline__ static int at(int x, int y, int z) { return (z * MY + y) * PX + x; }
  __device__ __forceinline__ static int at_flat(int i) {
    int x = i % MX, r = i / MX;
    return r * PX + x;  // r = z * MY + y
  }
};

// Line mappers: line index l -> base offset; element stride ESTR.  Consecutive l are
// consecutive x whenever x is not the transform axis, and consecutive rows otherwise.
template <class LY, int AXIS> struct Lines;
template <class LY> struct Lines<LY, 0> {  // along x
  static constexpr int M = LY::PX - 1;
  static constexpr int NL = LY::N / M;
  static constexpr int ESTR = 1;
  __device__ __forceinline__ static int base(int l) { return l * LY::PX; }
};
template <int MX, int MY, int MZ> struct Lines<Layout<MX, MY, MZ>, 1> {  // along y
  using LY = Layout<MX, MY, MZ>;
  static constexpr int M = MY;
  static constexpr int NL = MX * MZ;
  static constexpr int ESTR = LY::PX;
  __device__ __forceinline__ static int base(int l) { return (l / MX) * MY * LY::PX + (l % MX); }
};
template <int MX, int MY, int MZ> struct Lines<Layout<MX, MY, MZ>, 2> {  // along z
  using LY = Layout<MX, MY, MZ>;
  static constexpr int M = MZ;
  static constexpr int NL = MX * MY;
  static constexpr int ESTR = MY * LY::PX;
  __device__ __forceinline__ static int base(int l) { return (l / MX) * LY::PX + (l % MX); }
};

// Identity: the element-wise operation a pass applies to its inputs by default.
struct NoPre {
  template <typename C> __device__ __forceinline__ C operator()(C v, int, int) const { return v; }
};

// One in-place Stockham pass (radix R, NS = product of earlier radices).  pre(v, l, pos)
// is applied to every input as it is loaded (line l, position pos along the axis), so a
// point-wise multiplier can ride on the first pass of a transform.
template <int R, int NS, int SGN, class LN, int NT, typename C, class F = NoPre>
__device__ __forceinline__ void pass(C* s, const C* tw, F pre = F()) {
  constexpr int M = LN::M;
  constexpr int NBL = M / R;
  constexpr int NB = LN::NL * NBL;
  constexpr int PER = (NB + NT - 1) / NT;
  C v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = threadIdx.x + p * NT;
    if (NB % NT == 0 || b < NB) {
      const int l = b % LN::NL, j = b / LN::NL;
      const C* base = s + LN::base(l);
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = pre(base[(j + r * NBL) * LN::ESTR], l, j + r * NBL);
      if constexpr (NS > 1) {
        const int jm = j % NS;
        constexpr int STEP = M / (NS * R);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C t = tw[(r * jm * STEP) % M];
          if constexpr (SGN > 0) t = cconj(t);
          v[p][r] = cmul(v[p][r], t);
        }
      }
      dft<R, SGN>(v[p]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = threadIdx.x + p * NT;
    if (NB % NT == 0 || b < NB) {
      const int l = b % LN::NL, j = b / LN::NL;
      C* base = s + LN::base(l);
      const int idx = (j / NS) * NS * R + (j % NS);
#pragma unroll
      for (int r = 0; r < R; ++r) base[(idx + r * NS) * LN::ESTR] = v[p][r];
    }
  }
  __syncthreads();
}

// Full unnormalised DFT along one axis (SGN = -1 forward, +1 inverse); pre rides on the
// first pass.
template <int SGN, class LN, int NT, typename C, class F = NoPre>
__device__ __forceinline__ void axis(C* s, const C* tw, F pre = F()) {
  using P = Plan<LN::M>;
  pass<P::r0, 1, SGN, LN, NT>(s, tw, pre);
  if constexpr (P::np > 1) pass<P::r1, P::r0, SGN, LN, NT>(s, tw);
  if constexpr (P::np > 2) pass<P::r2, P::r0 * P::r1, SGN, LN, NT>(s, tw);
  if constexpr (P::np > 3) pass<P::r3, P::r0 * P::r1 * P::r2, SGN, LN, NT>(s, tw);
}

// Forward / inverse transform of the whole grid (all axes).  pre rides on the first pass
// of the first axis (x forward; z, else y, inverse): pre(v, l, pos) with that axis's line
// index l and position pos.
template <int SGN, class LY, int MZ, int NT, typename C, class F = NoPre>
__device__ __forceinline__ void transform(C* s, const C* twx, const C* twy, const C* twz, F pre = F()) {
  if constexpr (SGN < 0) {
    axis<SGN, Lines<LY, 0>, NT>(s, twx, pre);
    axis<SGN, Lines<LY, 1>, NT>(s, twy);
    if constexpr (MZ > 1) axis<SGN, Lines<LY, 2>, NT>(s, twz);
  } else {
    if constexpr (MZ > 1) {
      axis<SGN, Lines<LY, 2>, NT>(s, twz, pre);
      axis<SGN, Lines<LY, 1>, NT>(s, twy);
    } else {
      axis<SGN, Lines<LY, 1>, NT>(s, twy, pre);
    }
    axis<SGN, Lines<LY, 0>, NT>(s, twx);
  }
}

__device__ __forceinline__ int signed_k(int i, int m) { return i < m / 2 ? i : i - m; }

}  // namespace fft
}  // namespace omm
