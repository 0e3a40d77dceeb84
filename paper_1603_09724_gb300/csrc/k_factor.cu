// Multifrontal LU of the sparsifying matrix P on the device (Sec. 3.2: P is factored by a
// sparse direct method in nested-dissection order; by the complexity count after eq. P
// this setup dominates the cost of the preconditioner).  One call per tree height, every
// front of the height and every pole in each launch (grid.y / grid.z = pole):
//   assemble: the front of node s is zeroed, the couplings of P among its own unknowns and
//             its boundary are written, P(j, j + o_t) = q_t + qg_t (V_{j+o_t} - l) (eq. P),
//             and its children's update matrices are added, child by child
//             (extend-add); for a 2D leaf the couplings to its halo are kept as well;
//   lu:       partial LU of the first ns rows / columns without pivoting; a pivot below
//             pivot_floor times the largest entry of its updated row is raised to that
//             size (static pivoting); the trailing nb x nb block becomes the update matrix;
//   inv:      L_SS^-1 and U_SS^-1, the top block of W_f and the left block of W_b, one
//             column per thread; the banded L and U of the 2D leaves;
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

// Right-looking elimination of the first ns pivots: step k takes the largest entry of row
// k (already updated by the pivots before it) for the static pivot test, then each warp
// updates whole rows below it, lanes along the row.
template <typename T>
__global__ void __launch_bounds__(FT) fa_lu(FactorArgs f, const int* __restrict__ nodes, cx_t<T>* fronts,
                                            double* pstats) {
  using C = cx_t<T>;
  const int s = nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int ns = f.node_ns[s], nf = ns + f.node_nb[s];
  C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = FT / 32;
  __shared__ T red[NW];
  __shared__ C s_ip;
  double pmin = DBL_MAX, pmax = 0.0;
  int npert = 0;
  for (int k = 0; k < ns; ++k) {
    C* rk = F + (size_t)k * nf;
    T mx = 0;
    for (int j = k + tid; j < nf; j += FT) mx = fmax(mx, cabsv(rk[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    if (tid == 0) {
      T rown = red[0];
      for (int w = 1; w < NW; ++w) rown = fmax(rown, red[w]);
      C piv = rk[k];
      const T ap = cabsv(piv);
      const T floor_ = (T)f.pivot_floor;
      if (ap < floor_ * rown || ap == (T)0) {
        const T mag = floor_ * (rown > (T)0 ? rown : (T)1);
        piv = ap > (T)0 ? mk<C>(piv.x / ap * mag, piv.y / ap * mag) : mk<C>(mag, 0);
        rk[k] = piv;
        ++npert;
      }
      pmin = fmin(pmin, (double)cabsv(piv));
      pmax = fmax(pmax, (double)cabsv(piv));
      s_ip = crecip(piv);
    }
    __syncthreads();
    const C ip = s_ip;
    for (int i = k + 1 + wid; i < nf; i += NW) {
      C* ri = F + (size_t)i * nf;
      const C fik = ri[k];
      if (fik.x == (T)0 && fik.y == (T)0) continue;   // (warp-uniform) a zero multiplier changes nothing
      const C l = cmul(fik, ip);
      for (int j = k + 1 + lane; j < nf; j += 32) ri[j] = csub(ri[j], cmul(l, rk[j]));
      __syncwarp();
      if (lane == 0) ri[k] = l;
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* ps = pstats + ((size_t)p * f.nnodes + s) * 3;
    ps[0] = pmin;
    ps[1] = pmax;
    ps[2] = (double)npert;
  }
}

// L_SS^-1 into W_f rows 0..ns-1 and U_SS^-1 into W_b columns 0..ns-1, one column j per
// thread (zeros outside the triangles); the banded data of a 2D leaf.
template <typename T>
__global__ void __launch_bounds__(FT) fa_inv(FactorArgs f, const int* __restrict__ nodes, const cx_t<T>* fronts,
                                             cx_t<T>* factor, cx_t<T>* leafv) {
  using C = cx_t<T>;
  const int s = nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int ns = f.node_ns[s], nb = f.node_nb[s], nf = ns + nb, kb = ns + nb;
  const C* F = fronts + (size_t)p * f.front_size + f.foff[s];
  C* wf = factor + (size_t)p * f.factor_size + f.node_wf[s];
  C* wb = factor + (size_t)p * f.factor_size + f.node_wb[s];
  const int tid = threadIdx.x;
  for (int j = tid; j < ns; j += FT) {
    // L Li = I (unit lower L): Li(i, j) = -sum_{k = j}^{i - 1} L(i, k) Li(k, j), i > j
    for (int i = 0; i < j; ++i) wf[(size_t)i * ns + j] = mk<C>(0, 0);
    wf[(size_t)j * ns + j] = mk<C>(1, 0);
    for (int i = j + 1; i < ns; ++i) {
      const C* li = F + (size_t)i * nf;
      C acc = mk<C>(0, 0);
      for (int k = j; k < i; ++k) acc = cfma(li[k], wf[(size_t)k * ns + j], acc);
      wf[(size_t)i * ns + j] = mk<C>(-acc.x, -acc.y);
    }
    // U Ui = I: Ui(i, j) = (delta_ij - sum_{k = i + 1}^{j} U(i, k) Ui(k, j)) / U(i, i), i <= j
    for (int i = ns - 1; i > j; --i) wb[(size_t)i * kb + j] = mk<C>(0, 0);
    wb[(size_t)j * kb + j] = crecip(F[(size_t)j * nf + j]);
    for (int i = j - 1; i >= 0; --i) {
      const C* ui = F + (size_t)i * nf;
      C acc = mk<C>(0, 0);
      for (int k = i + 1; k <= j; ++k) acc = cfma(ui[k], wb[(size_t)k * kb + j], acc);
      wb[(size_t)i * kb + j] = cmul(mk<C>(-acc.x, -acc.y), crecip(ui[i]));
    }
  }
  const int li = f.leaf_of[s];
  if (li < 0) return;
  const int bw = f.leaf_bw;
  C* Lb = leafv + (size_t)p * f.leaf_size + f.leaf_voff[li];
  C* Ub = Lb + (size_t)ns * bw;
  for (int e = tid; e < ns * bw; e += FT) {
    const int i = e / bw, j = i - 1 - e % bw;
    Lb[e] = j >= 0 ? F[(size_t)i * nf + j] : mk<C>(0, 0);
  }
  for (int e = tid; e < ns * (bw + 1); e += FT) {
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
  if (t >= 2 * tn * tb) return;
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
cudaError_t run_height(const FactorArgs& f, const int* nodes, int count, int P, int max_tiles, void* fronts,
                       void* factor, void* leafv, double* pstats, cudaStream_t st) {
  using C = cx_t<T>;
  if (count <= 0) return cudaSuccess;
  const dim3 g2(count, P);
  fa_assemble<T><<<g2, FT, 0, st>>>(f, nodes, (C*)fronts, (C*)leafv);
  fa_lu<T><<<g2, FT, 0, st>>>(f, nodes, (C*)fronts, pstats);
  fa_inv<T><<<g2, FT, 0, st>>>(f, nodes, (const C*)fronts, (C*)factor, (C*)leafv);
  if (max_tiles > 0) fa_wprod<T><<<dim3(max_tiles, count, P), FT, 0, st>>>(f, nodes, (const C*)fronts, (C*)factor);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_factor_height(const FactorArgs& f, const int* nodes, int count, int P, int max_tiles,
                                 double2* fronts, double2* factor, double2* leafv, double* pstats, cudaStream_t st) {
  if (P < 1 || P > 65535 || count > 65535) return cudaErrorInvalidValue;
  return run_height<double>(f, nodes, count, P, max_tiles, fronts, factor, leafv, pstats, st);
}

cudaError_t launch_factor_to_c64(const double2* src, float2* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((count + 255) / 256, 152 * 16);
  factor_to_c64<<<(unsigned)blocks, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

}  // namespace omm
