// Device triangular solves with the multifrontal factor of the sparsifying matrix P
// (Sec. 3.2: the preconditioned vector is P^-1 Q G b, and P is factored by a sparse
// direct method in nested-dissection order).  Unknowns are numbered in ND postorder;
// supernode s owns the contiguous range [off, off + ns) and couples to the ancestor
// unknowns B(s).  The right-hand side b arrives in ND order (the Green kernel stores it
// so), and every intermediate vector stays in ND order: y in ynd, the assembled
// separator right-hand sides and then the solution in xnd.  So every gather of the
// solves reads contiguous runs (a supernode's range, or the pieces of ancestor
// separators that form B(s)); only the final solution is also scattered into natural
// order (x) for the operators that follow.
//
// With W_f = [L_SS^-1 ; L_BS L_SS^-1] and W_b = [U_SS^-1 , -U_SS^-1 U_SB] (built on the
// host) every supernode step is one dense complex product over a tile of right-hand
// sides, with no sequential sweep:
//   forward  (leaves first):  [y_S ; u_s] = W_f (b_S - sum of the update rows u_D that
//            target S)            -- y_S kept in ND order, u_s for the ancestors
//   backward (root first):    x_S = W_b [y_S ; x_B]   -- x_B gathered from the ancestors
// Per tree height and direction: one assembly launch (forward only) and one product
// launch.  A product CTA computes RB = 64 rows of one supernode's product for RT
// right-hand sides of one pole (system s = p * N + c), with the right-hand-side block
// staged in shared memory and 4 x (RT/8) outputs per thread.  Leaves (height 0) use
// their banded LU instead of dense W blocks (leaf_kernel).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "trsv.h"

namespace omm {

template <typename T> struct TrsvCfg;
template <> struct TrsvCfg<float> { static constexpr int RT = 32; };
template <> struct TrsvCfg<double> { static constexpr int RT = 16; };
constexpr int RB = 64;   // rows per CTA
constexpr int KT = 16;   // k step of the product

// Forward right-hand sides of one tree height: r_S = b_S - (sum of the update rows of the
// descendants that target S, in CSR order), for every unknown of the height and every
// active system of the launch (nsys = its poles x N; u rows have stride a.S, the systems of
// all poles), written in ND order into xnd (the backward sweep later overwrites every
// entry of an active system with the solution).  An AS_I x 32 tile (unknowns x
// systems, one element per thread) is transposed through shared memory so that the
// reads of b and the store into xnd run unknown-fastest while the update rows are read
// system-fastest.  Small tiles: the top heights have few unknowns, and each element waits
// on a chain of loads, so the grid needs many CTAs.
constexpr int AS_I = 8;

// Update rows, ynd and xnd are read with ld.global.cg (L2, not the SM's L1): inside the
// persistent launch below, other SMs wrote them earlier in the same kernel.
template <typename T>
__device__ __forceinline__ void assemble_tile(const TrsvArgs& a, const int* __restrict__ lunk, int cnt, size_t nsys,
                                              const cx_t<T>* __restrict__ b, const cx_t<T>* u, cx_t<T>* x,
                                              const int* __restrict__ active, int bx, int by) {
  using C = cx_t<T>;
  __shared__ C tile[AS_I][33];
  const int i0 = bx * AS_I;
  const size_t s0 = (size_t)by * 32;
  const int t = threadIdx.x;
  {
    const int ii = t % AS_I, ss = t / AS_I;   // unknown fastest
    const int i = i0 + ii;
    const size_t s = s0 + ss;
    if (i < cnt && s < nsys && (!active || active[s])) tile[ii][ss] = b[s * a.n + lunk[i]];
  }
  __syncthreads();
  {
    const int ss = t % 32, ii = t / 32;       // system fastest
    const int i = i0 + ii;
    const size_t s = s0 + ss;
    if (i < cnt && s < nsys && (!active || active[s])) {
      const int nd = lunk[i];
      const int e0 = a.contrib_ptr[nd], e1 = a.contrib_ptr[nd + 1];
      C acc = tile[ii][ss];
      int e = e0;
      for (; e + 4 <= e1; e += 4) {   // four independent loads in flight, subtracted in order
        const C v0 = __ldcg(u + (size_t)a.contrib_idx[e] * a.S + s);
        const C v1 = __ldcg(u + (size_t)a.contrib_idx[e + 1] * a.S + s);
        const C v2 = __ldcg(u + (size_t)a.contrib_idx[e + 2] * a.S + s);
        const C v3 = __ldcg(u + (size_t)a.contrib_idx[e + 3] * a.S + s);
        acc = csub(csub(csub(csub(acc, v0), v1), v2), v3);
      }
      for (; e < e1; ++e) acc = csub(acc, __ldcg(u + (size_t)a.contrib_idx[e] * a.S + s));
      tile[ii][ss] = acc;
    }
  }
  __syncthreads();
  {
    const int ii = t % AS_I, ss = t / AS_I;
    const int i = i0 + ii;
    const size_t s = s0 + ss;
    if (i < cnt && s < nsys && (!active || active[s])) x[s * a.n + lunk[i]] = tile[ii][ss];
  }
}

template <typename T>
__global__ void __launch_bounds__(AS_I * 32) assemble_kernel(TrsvArgs a, const int* __restrict__ lunk, int cnt,
                                                              size_t nsys, const cx_t<T>* __restrict__ b,
                                                              const cx_t<T>* u, cx_t<T>* x, const int* __restrict__ active) {
  griddep_wait();
  griddep_launch();
  assemble_tile<T>(a, lunk, cnt, nsys, b, u, x, active, blockIdx.x, blockIdx.y);
}

// Grid: (right-hand-side tiles, row blocks, poles).  The tiles of one row block are
// adjacent in launch order, so the W rows they share are read from DRAM once.
// RBV rows x RTV right-hand sides per CTA with NTH threads, 4 rows x TC columns per thread.
// The host's row blocks are 64 rows; a smaller RBV splits each into `split` CTAs (grid.y):
// for the top of the tree, where 64-row blocks leave most SMs idle, and for thin nodes.
template <typename T, bool FWD, int RBV, int RTV, int NTH, bool GD = false>
__device__ __forceinline__ void gemm_tile(const TrsvArgs& a, const int* __restrict__ blocks, cx_t<T>* ynd, cx_t<T>* u,
                                          cx_t<T>* x, cx_t<T>* xnd, const cx_t<T>* __restrict__ factor,
                                          const int* __restrict__ active, int split, int bx, int by, int bz,
                                          unsigned char* smem_raw) {
  using C = cx_t<T>;
  constexpr int RT = RTV;
  constexpr int TC = RTV * (RBV / 4) / NTH;   // columns per thread
  constexpr int CG = RTV / TC;                // column groups
  C* Bs = reinterpret_cast<C*>(smem_raw);   // [K][RT]
  __shared__ C As[2][KT][RBV + 1];                 // double-buffered W tiles
  C(*Cs)[RT + 1] = reinterpret_cast<C(*)[RT + 1]>(smem_raw);   // output staging, reuses Bs after the product
  const int node = blocks[2 * (by / split)];
  const int r0 = blocks[2 * (by / split) + 1] + (by % split) * RBV;
  const int p = bz;
  const int c0 = bx * RT;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node];
  const int K = FWD ? ns : ns + nb;
  const int M = FWD ? ns + nb : ns;
  if (r0 >= M) return;   // a split past the node's last row (uniform over the CTA)
  const C* W = factor + (size_t)p * a.factor_size + (FWD ? a.node_wf[node] : a.node_wb[node]);
  const int tid = threadIdx.x;
  // W_f's top block L_SS^-1 is lower and W_b's left block U_SS^-1 upper triangular: the
  // products of this row block run over the k range [klo, khi) that can hold nonzeros
  const int klo = FWD ? 0 : r0;
  const int khi = (FWD && r0 + RBV <= ns) ? min(K, r0 + RBV) : K;
  // W tiles: each thread holds WPT elements of the next tile in registers while the
  // current tile is consumed from shared memory (one barrier per k step).  The first tile
  // is loaded before the wait on the previous launch (GD): the factor is not written there.
  constexpr int WPT = RBV * KT / NTH;
  C wreg[WPT];
  auto load_w = [&](int k0) {
#pragma unroll
    for (int q = 0; q < WPT; ++q) {
      const int idx = tid + q * NTH;
      const int kk = idx % KT, rr = idx / KT;   // k fastest: coalesced rows of W
      const int r = r0 + rr, k = k0 + kk;
      wreg[q] = (r < M && k < khi) ? W[(size_t)r * K + k] : mk<C>(0, 0);
    }
  };
  load_w(klo);
  if (GD) {
    griddep_wait();
    griddep_launch();
  }
  // ---- right-hand-side block, i fastest (contiguous runs of one system's column); FB
  // independent loads in flight per thread
  constexpr int FB = 8;
  const int boff = a.node_boff[node];
  const int Kr = khi - klo;   // staged rows klo .. khi-1 of the block (Bs keeps absolute rows)
  for (int base = tid; base < Kr * RT; base += FB * NTH) {
    C v[FB];
#pragma unroll
    for (int q = 0; q < FB; ++q) {
      const int idx = base + q * NTH;
      const int i = klo + idx % Kr, cc = idx / Kr;
      const int c = c0 + cc;
      v[q] = mk<C>(0, 0);
      if (idx < Kr * RT && c < a.N) {
        const size_t s = (size_t)p * a.N + c;
        if (FWD) {   // assembled by assemble_kernel into xnd
          if (!active || active[s]) v[q] = __ldcg(xnd + s * a.n + off + i);
        } else {     // y_S, then x_B from the ancestors' solutions (runs in ND order)
          v[q] = __ldcg((i < ns) ? ynd + s * a.n + off + i : xnd + s * a.n + a.bnd[boff + i - ns]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < FB; ++q) {
      const int idx = base + q * NTH;
      if (idx < Kr * RT) Bs[(klo + idx % Kr) * RT + idx / Kr] = v[q];
    }
  }
  __syncthreads();
  // ---- product: rows r0 .. r0 + RBV - 1 of W times Bs
  const int tr = tid / CG, tcg = tid % CG;   // RBV / 4 row groups x CG column groups
  C acc[4][TC];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) acc[i][j] = mk<C>(0, 0);
  int buf = 0;
  for (int k0 = klo; k0 < khi; k0 += KT, buf ^= 1) {
#pragma unroll
    for (int q = 0; q < WPT; ++q) {
      const int idx = tid + q * NTH;
      As[buf][idx % KT][idx / KT] = wreg[q];
    }
    __syncthreads();
    if (k0 + KT < khi) load_w(k0 + KT);
    const int kmax = min(KT, khi - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      C av[4], bv[TC];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[buf][kk][tr * 4 + i];
#pragma unroll
      for (int j = 0; j < TC; ++j) bv[j] = Bs[(k0 + kk) * RT + tcg * TC + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
    }
  }
  __syncthreads();   // everyone is done with Bs before it becomes the output stage
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) Cs[tr * 4 + i][tcg * TC + j] = acc[i][j];
  __syncthreads();
  const int rows = min(RBV, M - r0);
  if (FWD) {
    // y rows (ND order, rr fastest) and update rows (system fastest)
    const int ny = max(0, min(rows, ns - r0));
    for (int idx = tid; idx < ny * RT; idx += NTH) {
      const int rr = idx % ny, cc = idx / ny;
      const int c = c0 + cc;
      if (c < a.N) ynd[((size_t)p * a.N + c) * a.n + off + r0 + rr] = Cs[rr][cc];
    }
    const int uoff = a.node_uoff[node];
    for (int idx = tid; idx < (rows - ny) * RT; idx += NTH) {
      const int cc = idx % RT, rr = ny + idx / RT;
      const int c = c0 + cc;
      if (c < a.N) u[(size_t)(uoff + r0 + rr - ns) * a.S + (size_t)p * a.N + c] = Cs[rr][cc];
    }
  } else {
    for (int idx = tid; idx < rows * RT; idx += NTH) {
      const int rr = idx % rows, cc = idx / rows;
      const int c = c0 + cc;
      if (c >= a.N) continue;
      const size_t s = (size_t)p * a.N + c;
      if (active && !active[s]) continue;
      xnd[s * a.n + off + r0 + rr] = Cs[rr][cc];          // for the descendants' gathers
      x[s * a.n + a.perm[off + r0 + rr]] = Cs[rr][cc];    // the result, natural order
    }
  }
}

template <typename T, bool FWD, int RBV, int RTV, int NTH>
__global__ void __launch_bounds__(NTH) trsv_gemm_kernel(TrsvArgs a, const int* __restrict__ blocks, cx_t<T>* ynd,
                                                        cx_t<T>* u, cx_t<T>* x, cx_t<T>* xnd,
                                                        const cx_t<T>* __restrict__ factor,
                                                        const int* __restrict__ active, int split) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gemm_tile<T, FWD, RBV, RTV, NTH, true>(a, blocks, ynd, u, x, xnd, factor, active, split, blockIdx.x, blockIdx.y,
                                   blockIdx.z, smem_raw);
}


// Split-K product for the upper tree heights, where one pole's nodes give too few CTAs
// for the tiled kernel above to keep the SMs busy and each of its threads walks the
// whole inner dimension K alone.  A CTA of 32 * KS threads computes one RBS x 16 tile
// (rows x right-hand sides) of one node's product: warp w accumulates the slice
// [w * kw, (w + 1) * kw) of K over its own copy of the tile (4 rows x TCS columns per
// lane, W rows staged per warp in WK-wide chunks, the next chunk's loads in flight while
// the current one is used), and the KS partial tiles are summed in shared memory in a
// fixed order, so the result does not depend on timing.  Shared memory: the
// right-hand-side block Bs [K][16] (reused for the partial tiles) and the warp-private W
// chunks.
constexpr int SK_RT = 16;   // right-hand sides per CTA
constexpr int SK_WK = 8;    // k values per staged W chunk

template <typename T, int KS, int RBS>
size_t sk_smem_bytes(int K) {
  const size_t cs = sizeof(cx_t<T>);
  const size_t bs = std::max((size_t)K * SK_RT, (size_t)KS * RBS * (SK_RT + 1));
  return (bs + (size_t)KS * SK_WK * (RBS + 1)) * cs;
}

template <typename T, bool FWD, int KS, int RBS, bool GD = false>
__device__ __forceinline__ void gemm_sk_tile(const TrsvArgs& a, const int* __restrict__ blocks, cx_t<T>* ynd,
                                             cx_t<T>* u, cx_t<T>* x, cx_t<T>* xnd, const cx_t<T>* __restrict__ factor,
                                             const int* __restrict__ active, int split, int bx, int by, int bz,
                                             unsigned char* smem_raw) {
  using C = cx_t<T>;
  constexpr int NTH = 32 * KS;
  constexpr int RT = SK_RT;
  constexpr int TCS = RBS * RT / (32 * 4);   // columns per lane (4 rows per lane)
  constexpr int CGS = RT / TCS;              // column groups across a warp
  const int node = blocks[2 * (by / split)];
  const int r0 = blocks[2 * (by / split) + 1] + (by % split) * RBS;
  const int p = bz;
  const int c0 = bx * RT;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node];
  const int K = FWD ? ns : ns + nb;
  const int M = FWD ? ns + nb : ns;
  if (r0 >= M) return;   // a split past the node's last row (uniform over the CTA)
  C* Bs = reinterpret_cast<C*>(smem_raw);                                   // [K][RT]
  const size_t bs_elems = max((size_t)K * RT, (size_t)KS * RBS * (RT + 1));
  C* Wall = Bs + bs_elems;                                                   // [KS][WK][RBS + 1]
  const C* W = factor + (size_t)p * a.factor_size + (FWD ? a.node_wf[node] : a.node_wb[node]);
  const int tid = threadIdx.x;
  // ---- this warp's slice of K; its first W chunk is loaded before the wait on the
  // previous launch (GD): the factor is not written there
  const int w = tid >> 5, lane = tid & 31;
  const int rg = lane / CGS, cg = lane % CGS;
  // only the k range [klo, khi) of this row block can hold nonzeros (L_SS^-1 lower,
  // U_SS^-1 upper triangular); the warps split that range
  const int klo = FWD ? 0 : r0;
  const int khi = (FWD && r0 + RBS <= ns) ? min(K, r0 + RBS) : K;
  const int Kr = khi - klo;
  const int kw = (Kr + KS - 1) / KS;
  const int kb = klo + w * kw, ke = min(khi, kb + kw);
  C* Ws = Wall + (size_t)w * SK_WK * (RBS + 1);
  constexpr int WPL = RBS * SK_WK / 32;   // W values per lane per chunk
  C wv[WPL];
  auto load_w = [&](int k0) {
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
      const int idx = lane + 32 * q;
      const int kk = idx % SK_WK, rr = idx / SK_WK;   // k fastest: runs of one W row
      const int r = r0 + rr, k = k0 + kk;
      wv[q] = (r < M && k < ke) ? W[(size_t)r * K + k] : mk<C>(0, 0);
    }
  };
  if (kb < ke) load_w(kb);
  if (GD) {
    griddep_wait();
    griddep_launch();
  }
  // ---- right-hand-side block (i fastest: contiguous runs of one system's column), rows
  // klo .. khi-1 (Bs keeps absolute rows)
  constexpr int FB = 8;
  const int boff = a.node_boff[node];
  for (int base = tid; base < Kr * RT; base += FB * NTH) {
    C v[FB];
#pragma unroll
    for (int q = 0; q < FB; ++q) {
      const int idx = base + q * NTH;
      const int i = klo + idx % Kr, cc = idx / Kr;
      const int c = c0 + cc;
      v[q] = mk<C>(0, 0);
      if (idx < Kr * RT && c < a.N) {
        const size_t s = (size_t)p * a.N + c;
        if (FWD) {
          if (!active || active[s]) v[q] = __ldcg(xnd + s * a.n + off + i);
        } else {
          v[q] = __ldcg((i < ns) ? ynd + s * a.n + off + i : xnd + s * a.n + a.bnd[boff + i - ns]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < FB; ++q) {
      const int idx = base + q * NTH;
      if (idx < Kr * RT) Bs[(klo + idx % Kr) * RT + idx / Kr] = v[q];
    }
  }
  __syncthreads();
  C acc[4][TCS];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TCS; ++j) acc[i][j] = mk<C>(0, 0);
  for (int k0 = kb; k0 < ke; k0 += SK_WK) {
    __syncwarp();   // the previous chunk has been read
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
      const int idx = lane + 32 * q;
      Ws[(idx % SK_WK) * (RBS + 1) + idx / SK_WK] = wv[q];
    }
    __syncwarp();
    if (k0 + SK_WK < ke) load_w(k0 + SK_WK);   // next chunk in flight during the products
    const int kmax = min(SK_WK, ke - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      C av[4], bv[TCS];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Ws[kk * (RBS + 1) + rg * 4 + i];
#pragma unroll
      for (int j = 0; j < TCS; ++j) bv[j] = Bs[(k0 + kk) * RT + cg * TCS + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TCS; ++j) acc[i][j] = cfma(av[i], bv[j], acc[i][j]);
    }
  }
  // ---- partial tiles -> Bs region [KS][RBS][RT + 1], summed in warp order into slice 0
  __syncthreads();   // every warp is done with Bs
  C* Rp = Bs;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TCS; ++j) Rp[((size_t)w * RBS + rg * 4 + i) * (RT + 1) + cg * TCS + j] = acc[i][j];
  __syncthreads();
  for (int o = tid; o < RBS * RT; o += NTH) {
    const int rr = o / RT, cc = o % RT;
    C sum = Rp[(size_t)rr * (RT + 1) + cc];
#pragma unroll
    for (int ww = 1; ww < KS; ++ww) sum = cadd(sum, Rp[((size_t)ww * RBS + rr) * (RT + 1) + cc]);
    Rp[(size_t)rr * (RT + 1) + cc] = sum;
  }
  __syncthreads();
  const int rows = min(RBS, M - r0);
  if (FWD) {
    const int ny = max(0, min(rows, ns - r0));
    for (int idx = tid; idx < ny * RT; idx += NTH) {
      const int rr = idx % ny, cc = idx / ny;
      const int c = c0 + cc;
      if (c < a.N) ynd[((size_t)p * a.N + c) * a.n + off + r0 + rr] = Rp[(size_t)rr * (RT + 1) + cc];
    }
    const int uoff = a.node_uoff[node];
    for (int idx = tid; idx < (rows - ny) * RT; idx += NTH) {
      const int cc = idx % RT, rr = ny + idx / RT;
      const int c = c0 + cc;
      if (c < a.N) u[(size_t)(uoff + r0 + rr - ns) * a.S + (size_t)p * a.N + c] = Rp[(size_t)rr * (RT + 1) + cc];
    }
  } else {
    for (int idx = tid; idx < rows * RT; idx += NTH) {
      const int rr = idx % rows, cc = idx / rows;
      const int c = c0 + cc;
      if (c >= a.N) continue;
      const size_t s = (size_t)p * a.N + c;
      if (active && !active[s]) continue;
      const C v = Rp[(size_t)rr * (RT + 1) + cc];
      xnd[s * a.n + off + r0 + rr] = v;
      x[s * a.n + a.perm[off + r0 + rr]] = v;
    }
  }
}

template <typename T, bool FWD, int KS, int RBS>
__global__ void __launch_bounds__(32 * KS) trsv_gemm_sk_kernel(TrsvArgs a, const int* __restrict__ blocks,
                                                               cx_t<T>* ynd, cx_t<T>* u, cx_t<T>* x, cx_t<T>* xnd,
                                                               const cx_t<T>* __restrict__ factor,
                                                               const int* __restrict__ active, int split) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  gemm_sk_tile<T, FWD, KS, RBS, true>(a, blocks, ynd, u, x, xnd, factor, active, split, blockIdx.x, blockIdx.y, blockIdx.z,
                                smem_raw);
}


// ---- leaves: banded substitution with the leaf's own L and U (the fill of a leaf stays
// inside the band of its x-fastest ordering) and sparse couplings to the halo:
//   forward:  y = L^-1 b_S,  u_s = F_BS (U^-1 y)       (b_S: a contiguous ND range)
//   backward: x_S = U^-1 (y_S - L^-1 (F_SB x_B))      (x_B from xnd, x_S stored in natural order)
// A CTA holds LT right-hand sides of one pole and one leaf in shared memory, column cc
// at y[i * LDY + cc], together with the leaf's factor values and index lists, staged
// once per CTA.  Global accesses are cooperative, leaf index fastest (a warp touches
// whole x-runs of one system's column), each one load behind an index already in shared
// memory; only the substitutions run one thread per right-hand side, on shared memory.
constexpr int LT = 128;       // right-hand sides per CTA for the leaves
constexpr int LDY = LT + 1;   // padded stride: the leaf-index-fastest accesses hit distinct banks
constexpr int LNB = 9;        // couplings per row of F_BS / F_SB (3^2 stencil)
constexpr int LGB = 8;        // gathered loads in flight per thread

// Band substitutions, one right-hand side per thread on its column of y (stride LDY).
// The band loops are unrolled to kMaxBw with the rows near the ends predicated, and each
// term is two fused multiply-adds per component (acc - l y), so a row costs about 4 bw FMA
// instructions and no loop control.  The last kMaxBw solved values stay in registers: the
// rows are unrolled in groups of kMaxBw, so row i of a group keeps its value in slot
// (i - first row) of the window and reads its neighbours' values from fixed slots.
constexpr int kMaxBw = 9;   // leaves of at most 8 x 8 points (x-fastest order: band <= 9)

template <typename C>
__device__ __forceinline__ C cfms(C l, C y, C acc) {   // acc - l * y
  acc.x = fma(-l.x, y.x, fma(l.y, y.y, acc.x));
  acc.y = fma(-l.x, y.y, fma(-l.y, y.x, acc.y));
  return acc;
}

template <typename T>
__device__ __forceinline__ void band_lower(cx_t<T>* y, int ns, int bw, const cx_t<T>* Lb) {
  using C = cx_t<T>;
  C win[kMaxBw];   // win[(i - i0) % kMaxBw] = y_i
  for (int i0 = 0; i0 < ns; i0 += kMaxBw) {
#pragma unroll
    for (int r = 0; r < kMaxBw; ++r) {
      const int i = i0 + r;
      if (i < ns) {
        C acc = y[i * LDY];
        const C* lr = Lb + i * bw;
        const int tn = min(bw, i);
#pragma unroll
        for (int t = 0; t < kMaxBw; ++t)   // y_{i-1-t} sits in slot (r - 1 - t) mod kMaxBw
          if (t < tn) acc = cfms(lr[t], win[(r - 1 - t + 2 * kMaxBw) % kMaxBw], acc);
        win[r] = acc;
        y[i * LDY] = acc;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void band_upper(cx_t<T>* y, int ns, int bw, const cx_t<T>* Ub) {
  using C = cx_t<T>;
  C win[kMaxBw];   // win[(i1 - i) % kMaxBw] = x_i, rows taken downwards from i1
  for (int i1 = ns - 1; i1 >= 0; i1 -= kMaxBw) {
#pragma unroll
    for (int r = 0; r < kMaxBw; ++r) {
      const int i = i1 - r;
      if (i >= 0) {
        C acc = y[i * LDY];
        const C* ur = Ub + i * (bw + 1);
        const int tn = min(bw, ns - 1 - i);
#pragma unroll
        for (int t = 1; t <= kMaxBw; ++t)   // x_{i+t} sits in slot (r - t) mod kMaxBw
          if (t <= tn) acc = cfms(ur[t], win[(r - t + 2 * kMaxBw) % kMaxBw], acc);
        acc = cmul(ur[0], acc);
        win[r] = acc;
        y[i * LDY] = acc;
      }
    }
  }
}

// shared memory of one leaf CTA: y block, the leaf's values, the halo values of 32
// columns (backward, stride LHS), its index lists
constexpr int LHS = 33;
__host__ __device__ inline size_t leaf_vals_count(int ns, int nb, int bw) {
  return (size_t)ns * bw + (size_t)ns * (bw + 1) + (size_t)nb * LNB + (size_t)ns * LNB;
}
__host__ __device__ inline size_t leaf_idx_count(int ns, int nb) { return (size_t)ns + nb + (size_t)(ns + nb) * LNB; }

template <typename T>
size_t leaf_smem_bytes(int max_ns, int max_nb, int bw) {
  return ((size_t)max_ns * LDY + leaf_vals_count(max_ns, max_nb, bw) + (size_t)max_nb * LHS) * sizeof(cx_t<T>) +
         leaf_idx_count(max_ns, max_nb) * sizeof(int);
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(LT) leaf_kernel(TrsvArgs a, LeafArgs la, const cx_t<T>* __restrict__ b,
                                                  cx_t<T>* __restrict__ ynd, cx_t<T>* __restrict__ u,
                                                  cx_t<T>* __restrict__ x, const cx_t<T>* __restrict__ xnd,
                                                  const int* __restrict__ active) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned char live[LT];
  const int li = blockIdx.y;
  const int node = la.nodes[li];
  const int p = blockIdx.z;
  const int c0 = blockIdx.x * LT;
  const int tid = threadIdx.x;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node];
  const int bw = la.bw;
  C* ys = reinterpret_cast<C*>(smem_raw);                                    // [ns][LDY]
  C* vs = ys + (size_t)la.max_ns * LDY;                                       // Lb | Ub | Fbs | Fsb
  C* hs = vs + leaf_vals_count(la.max_ns, la.max_nb, bw);                   // [max_nb][LHS]
  int* is = reinterpret_cast<int*>(hs + (size_t)la.max_nb * LHS);
  int* iperm = is;                  // natural index of leaf unknown i
  int* ibnd = iperm + ns;           // ND index of halo unknown j
  int* ibs = ibnd + nb;            // F_BS columns (leaf unknowns) per halo row, -1 padded
  int* isb = ibs + nb * LNB;        // F_SB columns (halo unknowns) per leaf row, -1 padded
  {   // the leaf's factor values and index lists (not written by the kernels before this one)
    const C* v = reinterpret_cast<const C*>(la.vals) + (size_t)p * la.leaf_size + la.voff[li];
    const int nv = (int)leaf_vals_count(ns, nb, bw);
    for (int e = tid; e < nv; e += LT) vs[e] = v[e];
    for (int i = tid; i < ns; i += LT) iperm[i] = a.perm[off + i];
    if (FWD) {
      const int* bsi = la.bs_idx + la.ioff_bs[li];
      for (int e = tid; e < nb * LNB; e += LT) ibs[e] = bsi[e];
    } else {
      const int boff = a.node_boff[node];
      const int* sbi = la.sb_idx + la.ioff_sb[li];
      for (int j = tid; j < nb; j += LT) ibnd[j] = a.bnd[boff + j];
      for (int e = tid; e < ns * LNB; e += LT) isb[e] = sbi[e];
    }
  }
  griddep_wait();
  griddep_launch();
  {
    const int c = c0 + tid;
    live[tid] = (c < a.N) && (!active || active[(size_t)p * a.N + c]);
  }
  __syncthreads();
  const C* Lb = vs;
  const C* Ub = Lb + ns * bw;
  const C* Fbs = Ub + ns * (bw + 1);
  const C* Fsb = Fbs + nb * LNB;
  const size_t s0 = (size_t)p * a.N + c0;
  C* y = ys + tid;
  const bool mine = live[tid];
  // Column passes between global memory and ys: warp wq takes the columns wq, wq + NWQ,
  // ... and its lanes consecutive leaf unknowns (i0 + lane, i0 + lane + 32), so that a
  // warp's accesses are contiguous runs of one column and no index needs a division.
  const int lane = tid & 31, wq = tid >> 5;
  constexpr int NWQ = LT / 32;
  static_assert(LT % (NWQ * LGB) == 0, "column batches tile the CTA");
  if (FWD) {
    for (int i0 = 0; i0 < ns; i0 += 64)
      for (int cb = wq; cb < LT; cb += NWQ * LGB) {   // 2 x LGB independent loads in flight
        C v[LGB][2];
#pragma unroll
        for (int q = 0; q < LGB; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = cb + q * NWQ, i = i0 + lane + 32 * h;
            if (i < ns && live[cc]) v[q][h] = b[(s0 + cc) * a.n + off + i];
          }
#pragma unroll
        for (int q = 0; q < LGB; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = cb + q * NWQ, i = i0 + lane + 32 * h;
            if (i < ns && live[cc]) ys[i * LDY + cc] = v[q][h];
          }
      }
    __syncthreads();
    if (mine) band_lower<T>(y, ns, bw, Lb);
    __syncthreads();
    for (int i0 = 0; i0 < ns; i0 += 64)
      for (int cc = wq; cc < LT; cc += NWQ) {
        if (!live[cc]) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = i0 + lane + 32 * h;
          if (i < ns) ynd[(s0 + cc) * a.n + off + i] = ys[i * LDY + cc];
        }
      }
    __syncthreads();
    if (!mine) return;
    band_upper<T>(y, ns, bw, Ub);
    const int uoff = a.node_uoff[node];
    for (int j = 0; j < nb; ++j) {   // system fastest across the CTA: coalesced update rows
      C acc = mk<C>(0, 0);
#pragma unroll
      for (int t = 0; t < LNB; ++t) {
        const int i = ibs[j * LNB + t];
        if (i < 0) break;   // the -1 padding trails: a halo row couples to few leaf unknowns
        acc = cfma(Fbs[j * LNB + t], y[i * LDY], acc);
      }
      u[(size_t)(uoff + j) * a.S + s0 + tid] = acc;
    }
  } else {
    // F_SB x_B, 32 columns at a time: the chunk's halo values are staged in shared memory
    // (lanes along the halo unknowns, which lie in runs of the ND order), then each warp
    // takes rows and its lanes the chunk's columns
    for (int cb = 0; cb < LT; cb += 32) {
      for (int c = wq; c < 32; c += NWQ) {
        const bool on = live[cb + c];
        const C* xs = xnd + (s0 + cb + c) * a.n;
        for (int j = lane; j < nb; j += 32) hs[j * LHS + c] = on ? xs[ibnd[j]] : mk<C>(0, 0);
      }
      __syncthreads();
      for (int i = wq; i < ns; i += NWQ) {
        C acc = mk<C>(0, 0);
#pragma unroll
        for (int t = 0; t < LNB; ++t) {   // -1 entries trail: same order as a breaking loop
          const int j = isb[i * LNB + t];
          if (j < 0) break;   // interior leaf unknowns have no halo couplings at all
          acc = cfma(Fsb[i * LNB + t], hs[j * LHS + lane], acc);
        }
        if (live[cb + lane]) ys[i * LDY + cb + lane] = acc;
      }
      __syncthreads();
    }
    __syncthreads();
    if (mine) band_lower<T>(y, ns, bw, Lb);
    __syncthreads();
    for (int i0 = 0; i0 < ns; i0 += 64)
      for (int cb = wq; cb < LT; cb += NWQ * LGB) {
        C v[LGB][2];
#pragma unroll
        for (int q = 0; q < LGB; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = cb + q * NWQ, i = i0 + lane + 32 * h;
            if (i < ns && live[cc]) v[q][h] = ynd[(s0 + cc) * a.n + off + i];
          }
#pragma unroll
        for (int q = 0; q < LGB; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int cc = cb + q * NWQ, i = i0 + lane + 32 * h;
            if (i < ns && live[cc]) ys[i * LDY + cc] = csub(v[q][h], ys[i * LDY + cc]);
          }
      }
    __syncthreads();
    if (mine) band_upper<T>(y, ns, bw, Ub);
    __syncthreads();
    for (int i0 = 0; i0 < ns; i0 += 64)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + lane + 32 * h;
        if (i >= ns) continue;
        const int xi = iperm[i];
        for (int cc = wq; cc < LT; cc += NWQ)
          if (live[cc]) x[(s0 + cc) * a.n + xi] = ys[i * LDY + cc];
      }
  }
}

// Shared memory of the largest product launch: K = max_ns + max_nb right-hand-side rows.
size_t trsv_smem_bytes(bool dbl, int max_ns, int max_nb) {
  const int RT = dbl ? TrsvCfg<double>::RT : TrsvCfg<float>::RT;
  const size_t cs = dbl ? sizeof(double2) : sizeof(float2);
  const size_t stat = cs * (2 * (size_t)KT * (RB + 1));
  return std::max((size_t)(max_ns + max_nb) * RT, (size_t)RB * (RT + 1)) * cs + stat;   // dynamic + static
}

template <typename T, bool FWD, int RBV, int RTV, int NTH>
static cudaError_t launch_level(const TrsvArgs& a, const int* blocks, int count, int kmax, int mmax, int P,
                                const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                                const int* active, bool ov, cudaStream_t st) {
  using C = cx_t<T>;
  auto k = trsv_gemm_kernel<T, FWD, RBV, RTV, NTH>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  // CTAs per 64-row host block: enough RBV-row tiles to cover min(64, mmax) rows
  const int split = (std::min(RB, mmax) + RBV - 1) / RBV;
  const dim3 grid((a.N + RTV - 1) / RTV, count * split, P);
  const size_t sm = std::max((size_t)kmax * RTV, (size_t)RBV * (RTV + 1)) * sizeof(C);
  (void)b;
  return launch_k(ov, k, grid, dim3(NTH), sm, st, a, blocks, (C*)ynd, (C*)u, (C*)x, (C*)xnd, (const C*)factor, active,
                  split);
}

// Tile choice per level from its largest row count mmax (M = ns + nb forward, ns backward)
// and its CTA count: 16-row tiles for the thin bottom separators (7 and 15 rows in 2D),
// 32 x RT/2 tiles where 64 x RT leaves the GPU underfilled, else 64 x RT.
template <typename T, bool FWD, int KS, int RBS>
static cudaError_t launch_level_sk(const TrsvArgs& a, const int* blocks, int count, int kmax, int mmax, int P,
                                   void* ynd, void* u, void* x, void* xnd, const void* factor, const int* active,
                                   bool ov, cudaStream_t st) {
  using C = cx_t<T>;
  auto k = trsv_gemm_sk_kernel<T, FWD, KS, RBS>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  const int split = (std::min(RB, mmax) + RBS - 1) / RBS;   // RBS-row CTAs per 64-row host block
  const dim3 grid((a.N + SK_RT - 1) / SK_RT, count * split, P);
  return launch_k(ov, k, grid, dim3(32 * KS), sk_smem_bytes<T, KS, RBS>(kmax), st, a, blocks, (C*)ynd, (C*)u,
                  (C*)x, (C*)xnd, (const C*)factor, active, split);
}

// Split-K launch for a level whose grid is small and whose inner dimension is long:
// 16-row tiles for nodes of at most 16 rows, else 32; 8 warps per CTA from K = 128, else 4.
template <typename T, bool FWD>
static bool try_level_sk(cudaError_t* err, const TrsvArgs& a, const int* blocks, int count, int kmax, int mmax,
                         int P, void* ynd, void* u, void* x, void* xnd, const void* factor, const int* active,
                         bool ov, cudaStream_t st) {
  if (kmax < 48) return false;
  const int KS = kmax >= 128 ? 8 : 4;
  const int RBS = mmax <= 16 ? 16 : 32;
  const size_t sm = KS == 8 ? (RBS == 16 ? sk_smem_bytes<T, 8, 16>(kmax) : sk_smem_bytes<T, 8, 32>(kmax))
                            : (RBS == 16 ? sk_smem_bytes<T, 4, 16>(kmax) : sk_smem_bytes<T, 4, 32>(kmax));
  if (sm > 200 * 1024) return false;
  if (KS == 8 && RBS == 16)
    *err = launch_level_sk<T, FWD, 8, 16>(a, blocks, count, kmax, mmax, P, ynd, u, x, xnd, factor, active, ov, st);
  else if (KS == 8)
    *err = launch_level_sk<T, FWD, 8, 32>(a, blocks, count, kmax, mmax, P, ynd, u, x, xnd, factor, active, ov, st);
  else if (RBS == 16)
    *err = launch_level_sk<T, FWD, 4, 16>(a, blocks, count, kmax, mmax, P, ynd, u, x, xnd, factor, active, ov, st);
  else
    *err = launch_level_sk<T, FWD, 4, 32>(a, blocks, count, kmax, mmax, P, ynd, u, x, xnd, factor, active, ov, st);
  return true;
}

template <typename T, bool FWD>
static cudaError_t run_level(const TrsvArgs& a, const int* blocks, int count, int kmax, int mmax, int P,
                             const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                             const int* active, bool ov, cudaStream_t st) {
  constexpr int RT = TrsvCfg<T>::RT;
  {
    // grids that leave most SMs idle with the tiled kernel: split K across warps instead
    const long tiled = (long)count * ((a.N + RT - 1) / RT) * P * ((std::min(RB, mmax) + 31) / 32);
    cudaError_t e = cudaSuccess;
    if (tiled < 4 * 152 && try_level_sk<T, FWD>(&e, a, blocks, count, kmax, mmax, P, ynd, u, x, xnd, factor,
                                                 active, ov, st))
      return e;
  }
  if (mmax <= 16)
    return launch_level<T, FWD, 16, RT, 64>(a, blocks, count, kmax, mmax, P, b, ynd, u, x, xnd, factor, active, ov, st);
  const long ctas = (long)count * ((a.N + RT - 1) / RT) * P;
  if (ctas >= 8 * 152 && mmax > 32)
    return launch_level<T, FWD, 64, RT, 128>(a, blocks, count, kmax, mmax, P, b, ynd, u, x, xnd, factor, active, ov, st);
  return launch_level<T, FWD, 32, RT / 2, 64>(a, blocks, count, kmax, mmax, P, b, ynd, u, x, xnd, factor, active, ov, st);
}

template <typename T>
static cudaError_t run_t(int phases, const TrsvArgs& a, const TrsvLevels& lv, const LeafArgs& la, int P,
                         const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                         const int* active, size_t smem_total, bool ov, cudaStream_t st) {
  using C = cx_t<T>;
  (void)smem_total;
  auto leaf_f = leaf_kernel<T, true>;
  auto leaf_b = leaf_kernel<T, false>;
  for (const void* f : {(const void*)leaf_f, (const void*)leaf_b}) {
    cudaError_t e = raise_smem_limit(f);
    if (e != cudaSuccess) return e;
  }
  const bool leaves = la.nleaves > 0;
  if (leaves && la.bw > kMaxBw) return cudaErrorInvalidValue;   // the unrolled band loops cover kMaxBw
  const size_t lsm = leaf_smem_bytes<T>(la.max_ns, la.max_nb, la.bw);
  const dim3 lgrid((a.N + LT - 1) / LT, la.nleaves, P);
  if (leaves && (phases & SPP_LEAF_FWD)) {
    cudaError_t e = launch_k(ov, leaf_f, lgrid, dim3(LT), lsm, st, a, la, (const C*)b, (C*)ynd, (C*)u, (C*)x,
                             (const C*)xnd, active);
    if (e != cudaSuccess) return e;
  }
  for (int h = leaves ? 1 : 0; h < lv.nlevels && (phases & SPP_LEVELS_FWD); ++h) {
    if (lv.fcount[h] == 0) continue;
    if (lv.ucount[h] > 0) {
      const size_t nsys = (size_t)P * a.N;   // systems of this launch (a.S is the row stride of u)
      const dim3 agrid((lv.ucount[h] + AS_I - 1) / AS_I, (unsigned)((nsys + 31) / 32));
      cudaError_t e = launch_k(ov, assemble_kernel<T>, agrid, dim3(AS_I * 32), 0, st, a, lv.lunk + lv.ustart[h],
                               lv.ucount[h], nsys, (const C*)b, (const C*)u, (C*)xnd, active);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = run_level<T, true>(a, lv.fblocks + 2 * lv.fstart[h], lv.fcount[h], lv.fkmax[h], lv.bkmax[h], P,
                                       b, ynd, u, x, xnd, factor, active, ov, st);
    if (e != cudaSuccess) return e;
  }
  for (int h = lv.nlevels - 1; h >= (leaves ? 1 : 0) && (phases & SPP_LEVELS_BWD); --h) {
    if (lv.bcount[h] == 0) continue;
    cudaError_t e = run_level<T, false>(a, lv.bblocks + 2 * lv.bstart[h], lv.bcount[h], lv.bkmax[h], lv.fkmax[h], P,
                                        b, ynd, u, x, xnd, factor, active, ov, st);
    if (e != cudaSuccess) return e;
  }
  if (leaves && (phases & SPP_LEAF_BWD))
    return launch_k(ov, leaf_b, lgrid, dim3(LT), lsm, st, a, la, (const C*)b, (C*)ynd, (C*)u, (C*)x, (const C*)xnd,
                    active);
  return cudaSuccess;
}

// ---- all supernode heights of one application in one cooperative launch
// The forward sweep (per height: assembly, then the product) and the backward sweep are a
// fixed sequence of phases; each phase is a grid of tiles (the same tiles the separate
// launches above use, for all poles of the launch at once), and a grid-wide barrier
// separates consecutive phases.  Every CTA of the cooperative launch is resident, so the
// barrier completes; its waits are still bounded (2 s by %globaltimer): on timeout, or
// when another CTA already gave up, the kernel sets err and returns.
enum TrsvPhaseType : int { PH_ASM = 0, PH_FWD_TILE, PH_FWD_SK16, PH_FWD_SK32, PH_BWD_TILE, PH_BWD_SK16, PH_BWD_SK32 };

struct TrsvPhase {
  int type;
  int dimx, dimy, dimz;   // tile grid (x fastest)
  int split;              // CTAs per 64-row host block (products)
  int off;                // into lunk (assembly) or the (node, row) pairs of the height (products)
  int cnt;                // unknowns of the height (assembly)
  int pad;
};
constexpr int kMaxPhases = 64;
struct TrsvPhaseList {
  int n;
  TrsvPhase ph[kMaxPhases];
};
constexpr int PT = 256;   // threads of the persistent CTA (8 warps)

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0] counts arrivals, bar[1] is the generation; bar[2] is the error flag.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    volatile unsigned* verr = bar + 2;
    bool ok = *verr == 0u;
    if (ok) {
      const unsigned g = *gen;
      __threadfence();
      if (atomicAdd(bar, 1u) + 1u == nblocks) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        const unsigned long long t0 = global_timer_ns();
        while (*gen == g) {
          if (*verr != 0u || global_timer_ns() - t0 > 2000000000ull) {
            ok = false;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    if (!ok) atomicExch(bar + 2, 1u);
    *ok_sh = ok ? 1 : 0;
  }
  __syncthreads();
  return *ok_sh != 0;
}

template <typename T>
__global__ void __launch_bounds__(PT, 2) trsv_levels_kernel(TrsvArgs a, TrsvPhaseList L, const int* __restrict__ fblocks,
                                                        const int* __restrict__ bblocks, const int* __restrict__ lunk,
                                                        size_t nsys, const cx_t<T>* __restrict__ b, cx_t<T>* ynd,
                                                        cx_t<T>* u, cx_t<T>* x, cx_t<T>* xnd,
                                                        const cx_t<T>* __restrict__ factor,
                                                        const int* __restrict__ active, unsigned* bar) {
  constexpr int RT = TrsvCfg<T>::RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int ok_sh;
  for (int q = 0; q < L.n; ++q) {
    const TrsvPhase d = L.ph[q];
    const int ntasks = d.dimx * d.dimy * d.dimz;
    for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
      const int bx = t % d.dimx, by = (t / d.dimx) % d.dimy, bz = t / (d.dimx * d.dimy);
      switch (d.type) {
        case PH_ASM: assemble_tile<T>(a, lunk + d.off, d.cnt, nsys, b, u, xnd, active, bx, by); break;
        case PH_FWD_TILE:
          gemm_tile<T, true, 64, RT, PT>(a, fblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                         smem_raw);
          break;
        case PH_FWD_SK16:
          gemm_sk_tile<T, true, 8, 16>(a, fblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                       smem_raw);
          break;
        case PH_FWD_SK32:
          gemm_sk_tile<T, true, 8, 32>(a, fblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                       smem_raw);
          break;
        case PH_BWD_TILE:
          gemm_tile<T, false, 64, RT, PT>(a, bblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                          smem_raw);
          break;
        case PH_BWD_SK16:
          gemm_sk_tile<T, false, 8, 16>(a, bblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                        smem_raw);
          break;
        default:
          gemm_sk_tile<T, false, 8, 32>(a, bblocks + d.off, ynd, u, x, xnd, factor, active, d.split, bx, by, bz,
                                        smem_raw);
          break;
      }
      __syncthreads();   // shared memory is reused by the next tile
    }
    if (q + 1 < L.n && !grid_barrier(bar, gridDim.x, &ok_sh)) return;
  }
}

// Phase list and dynamic shared memory of the persistent launch; false if a phase does not
// fit (more phases than kMaxPhases, or tiles beyond 200 KB of shared memory).
template <typename T>
static bool build_phases(const TrsvArgs& a, const TrsvLevels& lv, bool leaves, int P, TrsvPhaseList& L, size_t& dyn) {
  constexpr int RT = TrsvCfg<T>::RT;
  const size_t cs = sizeof(cx_t<T>);
  const size_t nsys = (size_t)P * a.N;
  L.n = 0;
  dyn = 0;
  auto push = [&](TrsvPhase p) {
    if (L.n >= kMaxPhases) return false;
    L.ph[L.n++] = p;
    return true;
  };
  auto product = [&](bool fwd, int h) {
    const int kmax = fwd ? lv.fkmax[h] : lv.bkmax[h];
    const int mmax = fwd ? lv.bkmax[h] : lv.fkmax[h];
    TrsvPhase p{};
    p.off = 2 * (fwd ? lv.fstart[h] : lv.bstart[h]);
    const int count = fwd ? lv.fcount[h] : lv.bcount[h];
    if (kmax >= 48) {
      const int RBS = mmax <= 16 ? 16 : 32;
      p.type = fwd ? (RBS == 16 ? PH_FWD_SK16 : PH_FWD_SK32) : (RBS == 16 ? PH_BWD_SK16 : PH_BWD_SK32);
      p.split = (std::min(RB, mmax) + RBS - 1) / RBS;
      p.dimx = (a.N + SK_RT - 1) / SK_RT;
      dyn = std::max(dyn, RBS == 16 ? sk_smem_bytes<T, 8, 16>(kmax) : sk_smem_bytes<T, 8, 32>(kmax));
    } else {
      p.type = fwd ? PH_FWD_TILE : PH_BWD_TILE;
      p.split = 1;
      p.dimx = (a.N + RT - 1) / RT;
      dyn = std::max(dyn, std::max((size_t)kmax * RT, (size_t)RB * (RT + 1)) * cs);
    }
    p.dimy = count * p.split;
    p.dimz = P;
    return push(p);
  };
  const int h0 = leaves ? 1 : 0;
  for (int h = h0; h < lv.nlevels; ++h) {
    if (lv.fcount[h] == 0) continue;
    if (lv.ucount[h] > 0) {
      TrsvPhase p{};
      p.type = PH_ASM;
      p.dimx = (lv.ucount[h] + AS_I - 1) / AS_I;
      p.dimy = (int)((nsys + 31) / 32);
      p.dimz = 1;
      p.off = lv.ustart[h];
      p.cnt = lv.ucount[h];
      if (!push(p)) return false;
    }
    if (!product(true, h)) return false;
  }
  for (int h = lv.nlevels - 1; h >= h0; --h) {
    if (lv.bcount[h] == 0) continue;
    if (!product(false, h)) return false;
  }
  return L.n > 0 && dyn <= 200 * 1024;
}

template <typename T>
static cudaError_t run_levels_persistent(const TrsvArgs& a, const TrsvLevels& lv, bool leaves, int P, const void* b,
                                         void* ynd, void* u, void* x, void* xnd, const void* factor,
                                         const int* active, unsigned* bar, cudaStream_t st, bool* done) {
  using C = cx_t<T>;
  *done = false;
  static TrsvPhaseList L;   // host staging of the kernel argument (copied at launch)
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  size_t dyn = 0;
  if (!build_phases<T>(a, lv, leaves, P, L, dyn)) return cudaSuccess;
  auto k = trsv_levels_kernel<T>;
  cudaError_t e = raise_smem_limit((const void*)k);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, PT, dyn)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaSuccess;
  const dim3 grid((unsigned)(per_sm * sms));
  const size_t nsys = (size_t)P * a.N;
  const int* fb = lv.fblocks;
  const int* bb = lv.bblocks;
  const int* lu = lv.lunk;
  const C* bp = (const C*)b;
  C* yp = (C*)ynd;
  C* up = (C*)u;
  C* xp = (C*)x;
  C* xn = (C*)xnd;
  const C* fp = (const C*)factor;
  TrsvArgs aa = a;
  void* args[] = {&aa, &L, &fb, &bb, &lu, (void*)&nsys, &bp, &yp, &up, &xp, &xn, &fp, (void*)&active, &bar};
  e = cudaLaunchCooperativeKernel((const void*)k, grid, dim3(PT), args, dyn, st);
  if (e == cudaSuccess) *done = true;
  return e;
}

cudaError_t launch_spp_levels_persistent(bool dbl, const TrsvArgs& a, const TrsvLevels& lv, bool leaves, int P,
                                         const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                                         const int* active, unsigned* bar, cudaStream_t st, bool* done) {
  if (dbl) return run_levels_persistent<double>(a, lv, leaves, P, b, ynd, u, x, xnd, factor, active, bar, st, done);
  return run_levels_persistent<float>(a, lv, leaves, P, b, ynd, u, x, xnd, factor, active, bar, st, done);
}

cudaError_t launch_spp_solve(int phases, bool dbl, const TrsvArgs& a, const TrsvLevels& lv, const LeafArgs& la, int P,
                             const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                             const int* active, size_t smem, bool overlap, cudaStream_t st) {
  if (dbl) return run_t<double>(phases, a, lv, la, P, b, ynd, u, x, xnd, factor, active, smem, overlap, st);
  return run_t<float>(phases, a, lv, la, P, b, ynd, u, x, xnd, factor, active, smem, overlap, st);
}

}  // namespace omm
