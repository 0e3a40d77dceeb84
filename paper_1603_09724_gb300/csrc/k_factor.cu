// Multifrontal LU of the sparsifying matrix P on the device (Sec. 3.2: P is factored by a
// sparse direct method in nested-dissection order; by the complexity count after eq. P
// this setup dominates the cost of the preconditioner).  One call per tree height, every
// front of the height and every pole in each launch (grid.y / grid.z = pole):
//   assemble: the front of node s is zeroed, the couplings of P among its own unknowns and
//             its boundary are written, P(j, j + o_t) = q_t + qg_t (V_{j+o_t} - l) (eq. P),
//             and its children's update matrices are added, child by child
//             (extend-add); for a 2D leaf the couplings to its halo are kept as well;
//   lu:       partial LU of the first ns rows / columns without pivoting, in panels of 32
//             pivots (fa_panel) and rank-32 trailing updates over many CTAs (fa_trail); a
//             pivot below pivot_floor times the largest entry of its updated row is raised
//             to that size (static pivoting); the trailing nb x nb block becomes the
//             update matrix;
//   tinv:     L_SS^-1 and U_SS^-1, the top block of W_f and the left block of W_b, by
//             block rows of 32 (tiled products over the finished rows, then the block's
//             rows in order); the banded L and U of the 2D leaves (leafband);
//   wprod:    the rest of W_f = [L_SS^-1 ; L_BS L_SS^-1] and W_b = [U_SS^-1 , -U_SS^-1 U_SB]
//             as 32 x 32 output tiles.
// The steps are those of the host factorisation (host_spp.cpp), in FP64 (a complex64
// elimination loses up to three digits on the poles nearest the real axis); a mixed handle
// receives the factor rounded once to complex64 (factor_to_c64).
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "factor.h"

namespace omm {

namespace {

constexpr int FT = 256;   // threads per CTA

template <typename C>
__device__ __forceinline__ decltype(C::x) cabsv(C a) { return hypot(a.x, a.y); }

// 1 / a, scaled so that |a|^2 neither overflows nor underflows
template <typename C>
__device__ __forceinline__ C crecip(C a) {
  using T = decltype(C::x);
  const T s = fmax(fabs(a.x), fabs(a.y));
  const T xr = a.x / s, xi = a.y / s;
  const T d = (xr * xr + xi * xi) * s;
  return mk<C>(xr / d, -xi / d);
}

template <typename T>
__global__ void __launch_bounds__(FT) fa_assemble(FactorArgs f, const int* __restrict__ nodes, cx_t<T>* fronts,
                                                  cx_t<T>* leafv) {
  using C = cx_t<T>;
  const int s = nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int ns = f.node_ns[s], nb = f.node_nb[s], nf = ns + nb;
  C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  const int tid = threadIdx.x;
  for (size_t e = tid; e < (size_t)nf * nf; e += FT) F[e] = mk<C>(0, 0);
  __syncthreads();
  const double2* q = f.q + (size_t)p * f.na;
  const double2* qg = f.qg + (size_t)p * f.na;
  for (int k = f.asm_ptr[s] + tid; k < f.asm_ptr[s + 1]; k += FT) {
    const int src = f.asm_src[k];
    const int t = src % f.na;
    const double dv = f.V[f.nbr[src]] - f.lmean;
    F[f.asm_pos[k]] = mk<C>((T)(q[t].x + qg[t].x * dv), (T)(q[t].y + qg[t].y * dv));
  }
  const int li = f.leaf_of[s];
  if (li >= 0) {   // a leaf has no children: its front holds P's couplings only
    __syncthreads();
    constexpr int NB = 9;
    const int bw = f.leaf_bw;
    C* v = leafv + (size_t)p * f.leaf_size + f.leaf_voff[li];
    C* Fbs = v + (size_t)ns * bw + (size_t)ns * (bw + 1);
    C* Fsb = Fbs + (size_t)nb * NB;
    const int* bsi = f.leaf_bs_idx + f.leaf_ioff_bs[li];
    const int* sbi = f.leaf_sb_idx + f.leaf_ioff_sb[li];
    for (int e = tid; e < nb * NB; e += FT) {
      const int i = bsi[e];
      Fbs[e] = i >= 0 ? F[(size_t)(ns + e / NB) * nf + i] : mk<C>(0, 0);
    }
    for (int e = tid; e < ns * NB; e += FT) {
      const int j = sbi[e];
      Fsb[e] = j >= 0 ? F[(size_t)(e / NB) * nf + ns + j] : mk<C>(0, 0);
    }
    return;
  }
  for (int ci = 0; ci < 2; ++ci) {
    const int c = ci == 0 ? f.child0[s] : f.child1[s];
    if (c < 0) continue;
    __syncthreads();   // one child at a time, in the host's order
    const int nsc = f.node_ns[c], nbc = f.node_nb[c], nfc = nsc + nbc;
    const C* Fc = fronts + (size_t)p * f.front_size + f.foff[c];
    const int* em = f.emap + f.node_boff[c];
    for (int e = tid; e < nbc * nbc; e += FT) {
      const int a = e / nbc, b = e % nbc;
      C* d = F + (size_t)em[a] * nf + em[b];
      *d = cadd(*d, Fc[(size_t)(nsc + a) * nfc + nsc + b]);
    }
  }
}

// Blocked right-looking elimination of the first ns pivots, KP pivots per panel, in the
// order of the host's blocked LU (each element receives the same updates in the same
// order).  fa_panel, one CTA per front: for each pivot k of the panel, the part of row k
// right of the panel first receives the panel's earlier pivots; then the largest entry of
// the updated row k sets the static pivot test; then each thread computes the multiplier
// of a row below and updates that row's panel columns.  fa_trail: the
// rank-KP update of the trailing block right of and below the panel, 32 x 32 tiles over
// many CTAs.  Zero multipliers and zero entries of U are skipped (their products add
// nothing).
constexpr int KP = 32;

// The panel columns [kb, ke) of every row live in shared memory (stride KP + 1) when the
// front has at most PANEL_ROWS rows (SM), else they stay in global memory.  Step (c) gives
// each thread whole rows: the multiplier and the row's panel columns.
constexpr int PANEL_ROWS = 420;   // 420 x 33 x 16 B = 216.7 KB of shared memory

template <typename T, bool SM>
__device__ __forceinline__ void panel_body(const FactorArgs& f, cx_t<T>* F, int ns, int nf, int kb, double* ps,
                                           cx_t<T>* Ps) {
  using C = cx_t<T>;
  const int ke = min(kb + KP, ns), K = ke - kb;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = FT / 32;
  __shared__ T red[NW];
  __shared__ C s_ip;
  // panel entry (row i, column c), kb <= c < ke
  auto pan = [&](int i, int c) -> C& { return SM ? Ps[(size_t)i * (KP + 1) + (c - kb)] : F[(size_t)i * nf + c]; };
  if (SM) {
    for (int e = tid; e < nf * K; e += FT) {
      const int i = e / K, c = e % K;
      Ps[(size_t)i * (KP + 1) + c] = F[(size_t)i * nf + kb + c];
    }
    __syncthreads();
  }
  double pmin = DBL_MAX, pmax = 0.0;
  int npert = 0;
  for (int k = kb; k < ke; ++k) {
    C* rk = F + (size_t)k * nf;
    if (k > kb) {   // the part of row k right of the panel receives pivots kb .. k-1
      for (int j = ke + tid; j < nf; j += FT) {
        C acc = rk[j];
        for (int q = kb; q < k; ++q) {
          const C l = pan(k, q);
          if (l.x != (T)0 || l.y != (T)0) acc = csub(acc, cmul(l, F[(size_t)q * nf + j]));
        }
        rk[j] = acc;
      }
      __syncthreads();
    }
    T mx = 0;
    for (int j = k + tid; j < ke; j += FT) mx = fmax(mx, cabsv(pan(k, j)));
    for (int j = ke + tid; j < nf; j += FT) mx = fmax(mx, cabsv(rk[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    if (tid == 0) {
      T rown = red[0];
      for (int w = 1; w < NW; ++w) rown = fmax(rown, red[w]);
      C piv = pan(k, k);
      const T ap = cabsv(piv);
      const T floor_ = (T)f.pivot_floor;
      if (ap < floor_ * rown || ap == (T)0) {
        const T mag = floor_ * (rown > (T)0 ? rown : (T)1);
        piv = ap > (T)0 ? mk<C>(piv.x / ap * mag, piv.y / ap * mag) : mk<C>(mag, 0);
        pan(k, k) = piv;
        ++npert;
      }
      pmin = fmin(pmin, (double)cabsv(piv));
      pmax = fmax(pmax, (double)cabsv(piv));
      s_ip = crecip(piv);
    }
    __syncthreads();
    const C ip = s_ip;
    for (int i = k + 1 + tid; i < nf; i += FT) {   // one row per thread
      const C fik = pan(i, k);
      if (fik.x == (T)0 && fik.y == (T)0) continue;   // a zero multiplier changes nothing
      const C l = cmul(fik, ip);
      for (int j = k + 1; j < ke; ++j) {
        const C u = pan(k, j);
        if (u.x != (T)0 || u.y != (T)0) pan(i, j) = csub(pan(i, j), cmul(l, u));
      }
      pan(i, k) = l;
    }
    __syncthreads();
  }
  if (SM) {
    for (int e = tid; e < nf * K; e += FT) {
      const int i = e / K, c = e % K;
      F[(size_t)i * nf + kb + c] = Ps[(size_t)i * (KP + 1) + c];
    }
  }
  if (tid == 0) {
    if (kb == 0) {
      ps[0] = pmin;
      ps[1] = pmax;
      ps[2] = (double)npert;
    } else {
      ps[0] = fmin(ps[0], pmin);
      ps[1] = fmax(ps[1], pmax);
      ps[2] += (double)npert;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(FT) fa_panel(FactorArgs f, const int* __restrict__ nodes, cx_t<T>* fronts,
                                               double* pstats, int kb, int smem_rows) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char fa_smem[];
  const int s = nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int ns = f.node_ns[s], nf = ns + f.node_nb[s];
  if (kb >= ns) return;
  C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  double* ps = pstats + ((size_t)p * f.nnodes + s) * 3;
  if (nf <= smem_rows) panel_body<T, true>(f, F, ns, nf, kb, ps, reinterpret_cast<C*>(fa_smem));
  else panel_body<T, false>(f, F, ns, nf, kb, ps, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(FT) fa_trail(FactorArgs f, const int* __restrict__ nodes, cx_t<T>* fronts,
                                               int kb) {
  using C = cx_t<T>;
  __shared__ C As[32][KP + 1], Bs[KP][33];
  const int s = nodes[blockIdx.y];
  const int p = blockIdx.z;
  const int ns = f.node_ns[s], nf = ns + f.node_nb[s];
  if (kb >= ns) return;
  const int ke = min(kb + KP, ns), K = ke - kb;
  const int tm = (nf - ke + 31) / 32;
  const int t = blockIdx.x;
  if (t >= tm * tm) return;
  const int r0 = ke + (t / tm) * 32, c0 = ke + (t % tm) * 32;
  C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    As[rr][tx] = (r0 + rr < nf && tx < K) ? F[(size_t)(r0 + rr) * nf + kb + tx] : mk<C>(0, 0);
    Bs[rr][tx] = (rr < K && c0 + tx < nf) ? F[(size_t)(kb + rr) * nf + c0 + tx] : mk<C>(0, 0);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = r0 + ty + 8 * q, j = c0 + tx;
    if (i >= nf || j >= nf) continue;
    C acc = F[(size_t)i * nf + j];
    for (int kk = 0; kk < K; ++kk) {
      const C l = As[ty + 8 * q][kk];
      if (l.x != (T)0 || l.y != (T)0) acc = csub(acc, cmul(l, Bs[kk][tx]));   // (warp-uniform)
    }
    F[(size_t)i * nf + j] = acc;
  }
}

// L_SS^-1 into W_f rows 0..ns-1 and U_SS^-1 into W_b columns 0..ns-1 (zeros outside the
// triangles) by block rows of 32: launch b forms block row b of Li = L^-1 (top down) and
// block row nbk - 1 - b of Ui = U^-1 (bottom up), one 32 x 32 tile per CTA, from the block
// rows that earlier launches finished:
//   Li(r, c) = delta_rc - sum_{k < r} L(r, k) Li(k, c)          (unit lower L)
//   Ui(r, c) = (delta_rc - sum_{k > r} U(r, k) Ui(k, c)) / U(r, r)
// The sum over finished block rows is a tiled product (k restricted to where Li / Ui can
// be nonzero); the rows of the block then follow one after the other, one column per
// thread, with the block's diagonal tile of L or U in shared memory.  2D leaves are
// skipped (the solves use their banded data, fa_leafband).
template <typename T>
__global__ void __launch_bounds__(FT) fa_tinv(FactorArgs f, const int* __restrict__ nodes, const cx_t<T>* fronts,
                                              cx_t<T>* factor, int b) {
  using C = cx_t<T>;
  __shared__ C As[32][33], Bs[32][33], Ts[32][33];
  const int s = nodes[blockIdx.y];
  const int p = blockIdx.z;
  const int ns = f.node_ns[s], nb = f.node_nb[s], nf = ns + nb, kb = ns + nb;
  const int nbk = (ns + 31) / 32;
  if (f.leaf_of[s] >= 0 || b >= nbk || (int)blockIdx.x >= 2 * nbk) return;
  const bool lower = (int)blockIdx.x < nbk;
  const int c0 = 32 * (lower ? blockIdx.x : blockIdx.x - nbk);
  const int r0 = 32 * (lower ? b : nbk - 1 - b);
  const int rows = min(32, ns - r0), cols = min(32, ns - c0);
  const C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  C* X = factor + (size_t)p * f.factor_size + (lower ? f.node_wf[s] : f.node_wb[s]);
  const int ldx = lower ? ns : kb;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  // a tile strictly above (Li) or below (Ui) the diagonal is zero
  if ((lower && c0 >= r0 + 32) || (!lower && c0 + 32 <= r0)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      if (r < rows && tx < cols) X[(size_t)(r0 + r) * ldx + c0 + tx] = mk<C>(0, 0);
    }
    return;
  }
  C acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    acc[q] = mk<C>(r == c ? (T)1 : (T)0, 0);
  }
  // finished block rows that can couple: Li(k, c) = 0 for k < c, Ui(k, c) = 0 for k > c
  const int ka = lower ? c0 : r0 + 32, kz = lower ? r0 : min(ns, c0 + 32);
  for (int k0 = ka; k0 < kz; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = ty + 8 * q;
      const int ak = k0 + tx;
      As[rr][tx] = (rr < rows && ak < kz) ? F[(size_t)(r0 + rr) * nf + ak] : mk<C>(0, 0);
      const int bk = k0 + rr;
      Bs[rr][tx] = (bk < kz && tx < cols) ? X[(size_t)bk * ldx + c0 + tx] : mk<C>(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const C bv = Bs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = csub(acc[q], cmul(As[ty + 8 * q][kk], bv));
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    Ts[rr][tx] = acc[q];
    As[rr][tx] = (rr < rows && tx < rows) ? F[(size_t)(r0 + rr) * nf + r0 + tx] : mk<C>(0, 0);   // diagonal tile
  }
  __syncthreads();
  if (tid < 32 && tid < cols) {
    const int c = tid;
    if (lower) {
      for (int r = 1; r < rows; ++r) {
        C v = Ts[r][c];
        for (int kk = 0; kk < r; ++kk) v = csub(v, cmul(As[r][kk], Ts[kk][c]));
        Ts[r][c] = v;
      }
    } else {
      for (int r = rows - 1; r >= 0; --r) {
        C v = Ts[r][c];
        for (int kk = r + 1; kk < rows; ++kk) v = csub(v, cmul(As[r][kk], Ts[kk][c]));
        Ts[r][c] = cmul(v, crecip(As[r][r]));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    if (r < rows && tx < cols) X[(size_t)(r0 + r) * ldx + c0 + tx] = Ts[r][tx];
  }
}

// The banded L and U (inverted diagonal) of a 2D leaf from its factorised front.
template <typename T>
__global__ void __launch_bounds__(FT) fa_leafband(FactorArgs f, const int* __restrict__ nodes, const cx_t<T>* fronts,
                                                  cx_t<T>* leafv) {
  using C = cx_t<T>;
  const int s = nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int li = f.leaf_of[s];
  if (li < 0) return;
  const int ns = f.node_ns[s], nf = ns + f.node_nb[s];
  const C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  const int bw = f.leaf_bw;
  C* Lb = leafv + (size_t)p * f.leaf_size + f.leaf_voff[li];
  C* Ub = Lb + (size_t)ns * bw;
  for (int e = threadIdx.x; e < ns * bw; e += FT) {
    const int i = e / bw, j = i - 1 - e % bw;
    Lb[e] = j >= 0 ? F[(size_t)i * nf + j] : mk<C>(0, 0);
  }
  for (int e = threadIdx.x; e < ns * (bw + 1); e += FT) {
    const int i = e / (bw + 1), t = e % (bw + 1), j = i + t;
    Ub[e] = j < ns ? (t == 0 ? crecip(F[(size_t)i * nf + i]) : F[(size_t)i * nf + j]) : mk<C>(0, 0);
  }
}

// 32 x 32 output tiles of W_f's bottom block (nb x ns) = L_BS Li, then of W_b's right
// block (ns x nb) = -Ui U_SB; 256 threads, 4 outputs each, K in steps of 32 through
// shared memory.
template <typename T>
__global__ void __launch_bounds__(FT) fa_wprod(FactorArgs f, const int* __restrict__ nodes, const cx_t<T>* fronts,
                                               cx_t<T>* factor) {
  using C = cx_t<T>;
  __shared__ C As[32][33], Bs[32][33];
  const int s = nodes[blockIdx.y];
  const int p = blockIdx.z;
  const int ns = f.node_ns[s], nb = f.node_nb[s], nf = ns + nb, kb = ns + nb;
  const int tn = (ns + 31) / 32, tb = (nb + 31) / 32;
  int t = blockIdx.x;
  if (t >= 2 * tn * tb || f.leaf_of[s] >= 0) return;   // 2D leaves: banded data only
  const C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  C* wf = factor + (size_t)p * f.factor_size + f.node_wf[s];
  C* wb = factor + (size_t)p * f.factor_size + f.node_wb[s];
  const bool first = t < tn * tb;
  if (!first) t -= tn * tb;
  // first: A = L_BS (nb x ns, rows of F from ns), B = Li (ns x ns in wf), C = wf rows ns..
  // second: A = Ui (ns x ns in wb, ld kb), B = U_SB (ns x nb, F columns from ns), C = wb cols ns..
  const int M = first ? nb : ns, N = first ? ns : nb, K = ns;
  const int tcols = first ? tn : tb;
  const int r0 = (t / tcols) * 32, c0 = (t % tcols) * 32;
  const C* A = first ? F + (size_t)ns * nf : wb;
  const int lda = first ? nf : kb;
  const C* B = first ? wf : F + ns;
  const int ldb = first ? ns : nf;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  C acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = mk<C>(0, 0);
  for (int k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = ty + 8 * q;
      const int ar = r0 + rr, ak = k0 + tx;
      As[rr][tx] = (ar < M && ak < K) ? A[(size_t)ar * lda + ak] : mk<C>(0, 0);
      const int bk = k0 + rr, bc = c0 + tx;
      Bs[rr][tx] = (bk < K && bc < N) ? B[(size_t)bk * ldb + bc] : mk<C>(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const C b = Bs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = cfma(As[ty + 8 * q][kk], b, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r >= M || c >= N) continue;
    if (first) wf[(size_t)(ns + r) * ns + c] = acc[q];
    else wb[(size_t)r * kb + ns + c] = mk<C>(-acc[q].x, -acc[q].y);
  }
}

__global__ void factor_to_c64(const double2* __restrict__ src, float2* __restrict__ dst, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

template <typename T>
cudaError_t run_height(const FactorArgs& f, const FactorHeight& hh, int P, void* fronts, void* factor, void* leafv,
                       double* pstats, cudaStream_t st) {
  using C = cx_t<T>;
  if (hh.count <= 0) return cudaSuccess;
  const dim3 g2(hh.count, P);
  // shared memory for the panel columns of the height's largest stageable front
  const int prow = std::min(hh.max_nf, PANEL_ROWS);
  const size_t psm = (size_t)prow * (KP + 1) * sizeof(C);
  {
    cudaError_t e = raise_smem_limit((const void*)fa_panel<T>);
    if (e != cudaSuccess) return e;
  }
  fa_assemble<T><<<g2, FT, 0, st>>>(f, hh.nodes, (C*)fronts, (C*)leafv);
  for (int q = 0; q < hh.npanels; ++q) {
    fa_panel<T><<<g2, FT, psm, st>>>(f, hh.nodes, (C*)fronts, pstats, q * KP, prow);
    if (hh.trail_tiles[q] > 0)
      fa_trail<T><<<dim3(hh.trail_tiles[q], hh.count, P), FT, 0, st>>>(f, hh.nodes, (C*)fronts, q * KP);
  }
  if (hh.has_leaves) fa_leafband<T><<<g2, FT, 0, st>>>(f, hh.nodes, (const C*)fronts, (C*)leafv);
  const int nbk = (hh.max_ns + 31) / 32;
  if (hh.dense_nodes)
    for (int b = 0; b < nbk; ++b)
      fa_tinv<T><<<dim3(2 * nbk, hh.count, P), FT, 0, st>>>(f, hh.nodes, (const C*)fronts, (C*)factor, b);
  if (hh.wprod_tiles > 0)
    fa_wprod<T><<<dim3(hh.wprod_tiles, hh.count, P), FT, 0, st>>>(f, hh.nodes, (const C*)fronts, (C*)factor);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_factor_height(const FactorArgs& f, const FactorHeight& hh, int P, double2* fronts,
                                 double2* factor, double2* leafv, double* pstats, cudaStream_t st) {
  if (P < 1 || P > 65535 || hh.count > 65535 || hh.npanels < 0 || hh.npanels > FactorHeight::kMaxPanels)
    return cudaErrorInvalidValue;
  return run_height<double>(f, hh, P, fronts, factor, leafv, pstats, st);
}

cudaError_t launch_factor_to_c64(const double2* src, float2* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 16);
  factor_to_c64<<<(unsigned)blocks, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

}  // namespace omm
