// Device triangular solves with the multifrontal factor of the sparsifying matrix P
// (Sec. 3.2: u~ = P^-1 Q G b, "solved by sparse direct solvers such as nested
// dissection").  Unknowns are numbered in nested-dissection postorder; supernode s owns
// the contiguous range [off, off + ns) and couples to the ancestor unknowns B(s).
//
// With W_f = [L_SS^-1 ; L_BS L_SS^-1] and W_b = [U_SS^-1 , -U_SS^-1 U_SB] (built on the
// host) every supernode step is one dense complex product over a tile of right-hand
// sides, with no sequential sweep:
//   forward  (leaves first):  [y_S ; u_s] = W_f (b_S - sum of the update rows u_D that
//            target S)            -- y_S kept in ND order, u_s for the ancestors
//   backward (root first):    x_S = W_b [y_S ; x_B]   -- x_B gathered from the ancestors
// One launch per tree height and direction.  A CTA computes RB = 64 rows of one
// supernode's product for RT right-hand sides of one pole (system s = p * N + c), with
// the right-hand-side block staged in shared memory and 4 x (RT/8) outputs per thread.
#include <algorithm>

#include "common.cuh"
#include "trsv.h"

namespace omm {

template <typename T> struct TrsvCfg;
template <> struct TrsvCfg<float> { static constexpr int RT = 32; };
template <> struct TrsvCfg<double> { static constexpr int RT = 16; };
constexpr int TS_THREADS = 128;
constexpr int RB = 64;   // rows per CTA
constexpr int KT = 16;   // k step of the product

template <typename T, bool FWD>
__global__ void __launch_bounds__(TS_THREADS) trsv_gemm_kernel(TrsvArgs a, const int* __restrict__ blocks,
                                                               const cx_t<T>* __restrict__ b, cx_t<T>* __restrict__ ynd,
                                                               cx_t<T>* __restrict__ u, cx_t<T>* __restrict__ x,
                                                               const cx_t<T>* __restrict__ factor,
                                                               const int* __restrict__ active) {
  using C = cx_t<T>;
  constexpr int RT = TrsvCfg<T>::RT;
  constexpr int TC = RT / 8;   // columns per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Bs = reinterpret_cast<C*>(smem_raw);   // [K][RT]
  __shared__ C As[2][KT][RB + 1];                 // double-buffered W tiles
  C(*Cs)[RT + 1] = reinterpret_cast<C(*)[RT + 1]>(smem_raw);   // output staging, reuses Bs after the product
  const int node = blocks[2 * blockIdx.x], r0 = blocks[2 * blockIdx.x + 1];
  const int p = blockIdx.y;
  const int c0 = blockIdx.z * RT;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node];
  const int K = FWD ? ns : ns + nb;
  const int M = FWD ? ns + nb : ns;
  const C* W = factor + (size_t)p * a.factor_size + (FWD ? a.node_wf[node] : a.node_wb[node]);
  const int tid = threadIdx.x;
  // ---- right-hand-side block
  if (FWD) {
    for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {   // i fastest: coalesced along a line
      const int i = idx % ns, cc = idx / ns;
      const int c = c0 + cc;
      C v = mk<C>(0, 0);
      if (c < a.N) {
        const size_t s = (size_t)p * a.N + c;
        if (!active || active[s]) v = b[s * a.n + a.perm[off + i]];
      }
      Bs[i * RT + cc] = v;
    }
    __syncthreads();
    for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {   // cc fastest: u rows are [row][system]
      const int cc = idx % RT, i = idx / RT;
      const int c = c0 + cc;
      if (c >= a.N) continue;
      const size_t s = (size_t)p * a.N + c;
      const int e0 = a.contrib_ptr[off + i], e1 = a.contrib_ptr[off + i + 1];
      if (e0 == e1) continue;
      C acc = Bs[i * RT + cc];
      for (int e = e0; e < e1; ++e) acc = csub(acc, u[(size_t)a.contrib_idx[e] * a.S + s]);
      Bs[i * RT + cc] = acc;
    }
  } else {
    const int boff = a.node_boff[node];
    for (int idx = tid; idx < K * RT; idx += TS_THREADS) {
      const int i = idx % K, cc = idx / K;
      const int c = c0 + cc;
      C v = mk<C>(0, 0);
      if (c < a.N) {
        const size_t s = (size_t)p * a.N + c;
        v = (i < ns) ? ynd[s * a.n + off + i] : x[s * a.n + a.bnat[boff + i - ns]];
      }
      Bs[i * RT + cc] = v;
    }
  }
  __syncthreads();
  // ---- product: rows r0 .. r0 + RB - 1 of W times Bs
  const int tr = tid / 8, tcg = tid % 8;   // 16 row groups x 8 column groups
  C acc[4][TC];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) acc[i][j] = mk<C>(0, 0);
  // W tiles: each thread holds WPT elements of the next tile in registers while the
  // current tile is consumed from shared memory (one barrier per k step)
  constexpr int WPT = RB * KT / TS_THREADS;
  C wreg[WPT];
  auto load_w = [&](int k0) {
#pragma unroll
    for (int q = 0; q < WPT; ++q) {
      const int idx = tid + q * TS_THREADS;
      const int kk = idx % KT, rr = idx / KT;   // k fastest: coalesced rows of W
      const int r = r0 + rr, k = k0 + kk;
      wreg[q] = (r < M && k < K) ? W[(size_t)r * K + k] : mk<C>(0, 0);
    }
  };
  load_w(0);
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += KT, buf ^= 1) {
#pragma unroll
    for (int q = 0; q < WPT; ++q) {
      const int idx = tid + q * TS_THREADS;
      As[buf][idx % KT][idx / KT] = wreg[q];
    }
    __syncthreads();
    if (k0 + KT < K) load_w(k0 + KT);
    const int kmax = min(KT, K - k0);
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
  const int rows = min(RB, M - r0);
  if (FWD) {
    // y rows (ND order, rr fastest) and update rows (system fastest)
    const int ny = max(0, min(rows, ns - r0));
    for (int idx = tid; idx < ny * RT; idx += TS_THREADS) {
      const int rr = idx % ny, cc = idx / ny;
      const int c = c0 + cc;
      if (c < a.N) ynd[((size_t)p * a.N + c) * a.n + off + r0 + rr] = Cs[rr][cc];
    }
    const int uoff = a.node_uoff[node];
    for (int idx = tid; idx < (rows - ny) * RT; idx += TS_THREADS) {
      const int cc = idx % RT, rr = ny + idx / RT;
      const int c = c0 + cc;
      if (c < a.N) u[(size_t)(uoff + r0 + rr - ns) * a.S + (size_t)p * a.N + c] = Cs[rr][cc];
    }
  } else {
    for (int idx = tid; idx < rows * RT; idx += TS_THREADS) {
      const int rr = idx % rows, cc = idx / rows;
      const int c = c0 + cc;
      if (c >= a.N) continue;
      const size_t s = (size_t)p * a.N + c;
      if (active && !active[s]) continue;
      x[s * a.n + a.perm[off + r0 + rr]] = Cs[rr][cc];
    }
  }
}


// ---- leaves: one thread per right-hand side, the leaf's unknowns in a per-thread
// shared-memory column; banded substitution with the leaf's own L and U (the fill of a
// leaf stays inside the band of its x-fastest ordering), sparse couplings to the halo:
//   forward:  y = L^-1 b_S,  u_s = F_BS (U^-1 y)
//   backward: x_S = U^-1 (y_S - L^-1 (F_SB x_B))
constexpr int LT = 64;   // right-hand sides per CTA for the leaves

template <typename T>
__device__ __forceinline__ void band_lower(cx_t<T>* y, int ns, int bw, const cx_t<T>* Lb) {
  for (int i = 0; i < ns; ++i) {
    cx_t<T> acc = y[i * LT];
    const cx_t<T>* lr = Lb + (size_t)i * bw;
    for (int t = 0; t < bw; ++t) {
      const int j = i - 1 - t;
      if (j < 0) break;
      acc = csub(acc, cmul(lr[t], y[j * LT]));
    }
    y[i * LT] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void band_upper(cx_t<T>* y, int ns, int bw, const cx_t<T>* Ub) {
  for (int i = ns - 1; i >= 0; --i) {
    cx_t<T> acc = y[i * LT];
    const cx_t<T>* ur = Ub + (size_t)i * (bw + 1);
    for (int t = 1; t <= bw; ++t) {
      const int j = i + t;
      if (j >= ns) break;
      acc = csub(acc, cmul(ur[t], y[j * LT]));
    }
    y[i * LT] = cmul(ur[0], acc);
  }
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(LT) leaf_kernel(TrsvArgs a, LeafArgs la, const cx_t<T>* __restrict__ b,
                                                  cx_t<T>* __restrict__ ynd, cx_t<T>* __restrict__ u,
                                                  cx_t<T>* __restrict__ x, const int* __restrict__ active) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* y = reinterpret_cast<C*>(smem_raw) + threadIdx.x;   // element i at y[i * LT]
  const int li = blockIdx.x;
  const int node = la.nodes[li];
  const int p = blockIdx.y;
  const int c = blockIdx.z * LT + threadIdx.x;
  if (c >= a.N) return;
  const size_t s = (size_t)p * a.N + c;
  if (active && !active[s]) return;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node];
  const int bw = la.bw;
  constexpr int NB = 9;
  const C* v = reinterpret_cast<const C*>(la.vals) + (size_t)p * la.leaf_size + la.voff[li];
  const C* Lb = v;
  const C* Ub = Lb + (size_t)ns * bw;
  const C* Fbs = Ub + (size_t)ns * (bw + 1);
  const C* Fsb = Fbs + (size_t)nb * NB;
  if (FWD) {
    for (int i = 0; i < ns; ++i) y[i * LT] = b[s * a.n + a.perm[off + i]];
    band_lower<T>(y, ns, bw, Lb);
    for (int i = 0; i < ns; ++i) ynd[s * a.n + off + i] = y[i * LT];
    band_upper<T>(y, ns, bw, Ub);
    const int uoff = a.node_uoff[node];
    const int* bsi = la.bs_idx + la.ioff_bs[li];
    for (int j = 0; j < nb; ++j) {
      C acc = mk<C>(0, 0);
      for (int t = 0; t < NB; ++t) {
        const int i = bsi[j * NB + t];
        if (i < 0) break;
        acc = cfma(Fbs[(size_t)j * NB + t], y[i * LT], acc);
      }
      u[(size_t)(uoff + j) * a.S + s] = acc;
    }
  } else {
    const int boff = a.node_boff[node];
    const int* sbi = la.sb_idx + la.ioff_sb[li];
    for (int i = 0; i < ns; ++i) {
      C acc = mk<C>(0, 0);
      for (int t = 0; t < NB; ++t) {
        const int j = sbi[i * NB + t];
        if (j < 0) break;
        acc = cfma(Fsb[(size_t)i * NB + t], x[s * a.n + a.bnat[boff + j]], acc);
      }
      y[i * LT] = acc;
    }
    band_lower<T>(y, ns, bw, Lb);
    for (int i = 0; i < ns; ++i) y[i * LT] = csub(ynd[s * a.n + off + i], y[i * LT]);
    band_upper<T>(y, ns, bw, Ub);
    for (int i = 0; i < ns; ++i) x[s * a.n + a.perm[off + i]] = y[i * LT];
  }
}

size_t trsv_smem_bytes(bool dbl, int max_ns, int max_nb) {
  const int RT = dbl ? TrsvCfg<double>::RT : TrsvCfg<float>::RT;
  const size_t cs = dbl ? sizeof(double2) : sizeof(float2);
  const size_t stat = cs * (2 * (size_t)KT * (RB + 1));
  return std::max((size_t)(max_ns + max_nb) * RT, (size_t)RB * (RT + 1)) * cs + stat;   // dynamic + static
}

template <typename T>
static cudaError_t run_t(const TrsvArgs& a, const TrsvLevels& lv, const LeafArgs& la, int P, const void* b, void* ynd,
                         void* u, void* x, const void* factor, const int* active, size_t smem_total,
                         cudaStream_t st) {
  using C = cx_t<T>;
  constexpr int RT = TrsvCfg<T>::RT;
  (void)smem_total;
  for (const void* f : {(const void*)trsv_gemm_kernel<T, true>, (const void*)trsv_gemm_kernel<T, false>,
                        (const void*)leaf_kernel<T, true>, (const void*)leaf_kernel<T, false>}) {
    cudaError_t e = raise_smem_limit(f);
    if (e != cudaSuccess) return e;
  }
  const int tiles = (a.N + RT - 1) / RT;
  const bool leaves = la.nleaves > 0;
  const size_t lsm = (size_t)la.max_ns * LT * sizeof(C);
  const dim3 lgrid(la.nleaves, P, (a.N + LT - 1) / LT);
  if (leaves) {
    leaf_kernel<T, true><<<lgrid, LT, lsm, st>>>(a, la, (const C*)b, (C*)ynd, (C*)u, (C*)x, active);
  }
  // dynamic shared memory sized per level (the root fronts need ~100 KB)
  for (int h = leaves ? 1 : 0; h < lv.nlevels; ++h) {
    if (lv.fcount[h] == 0) continue;
    dim3 grid(lv.fcount[h], P, tiles);
    const size_t sm = (size_t)std::max(lv.fkmax[h] * RT, RB * (RT + 1)) * sizeof(C);
    trsv_gemm_kernel<T, true><<<grid, TS_THREADS, sm, st>>>(a, lv.fblocks + 2 * lv.fstart[h], (const C*)b, (C*)ynd,
                                                            (C*)u, (C*)x, (const C*)factor, active);
  }
  for (int h = lv.nlevels - 1; h >= (leaves ? 1 : 0); --h) {
    if (lv.bcount[h] == 0) continue;
    dim3 grid(lv.bcount[h], P, tiles);
    const size_t sm = (size_t)std::max(lv.bkmax[h] * RT, RB * (RT + 1)) * sizeof(C);
    trsv_gemm_kernel<T, false><<<grid, TS_THREADS, sm, st>>>(a, lv.bblocks + 2 * lv.bstart[h], (const C*)b, (C*)ynd,
                                                             (C*)u, (C*)x, (const C*)factor, active);
  }
  if (leaves) leaf_kernel<T, false><<<lgrid, LT, lsm, st>>>(a, la, (const C*)b, (C*)ynd, (C*)u, (C*)x, active);
  return cudaGetLastError();
}

cudaError_t launch_spp_solve(bool dbl, const TrsvArgs& a, const TrsvLevels& lv, const LeafArgs& la, int P,
                             const void* b, void* ynd, void* u, void* x, const void* factor, const int* active,
                             size_t smem, cudaStream_t st) {
  if (dbl) return run_t<double>(a, lv, la, P, b, ynd, u, x, factor, active, smem, st);
  return run_t<float>(a, lv, la, P, b, ynd, u, x, factor, active, smem, st);
}

}  // namespace omm
