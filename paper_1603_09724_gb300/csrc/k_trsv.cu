// Device triangular solves with the multifrontal factor of the sparsifying matrix P
// (Sec. 3.2: u~ = P^-1 Q G b, "solved by sparse direct solvers such as nested
// dissection").  Unknowns are numbered in nested-dissection postorder; each supernode s
// owns a contiguous range [off, off + ns) and a boundary list B(s) of ancestor unknowns.
//
// Forward (L y = b), leaves first, one launch per tree height:
//   y_S = b_S - sum of the update rows u_D that target S (deterministic gather)
//   y_S = L_SS^-1 y_S   (unit lower, column sweep with one barrier per column)
//   u_s = L_BS y_S      (update rows for the ancestors)
// Backward (U x = y), root first:
//   t = y_S - U_SB x_B  (x_B gathered from the ancestors' finished unknowns)
//   x_S = U_SS^-1 t     (upper, the diagonal stored inverted)
// A CTA handles one supernode of one pole for RT right-hand sides; b and x are in the
// natural grid order (gathered / scattered through the ND permutation), y is kept in ND
// order.  System s = p * N + c uses pole p's factor.
#include "common.cuh"
#include "trsv.h"

namespace omm {

template <typename T> struct TrsvCfg;
template <> struct TrsvCfg<float> { static constexpr int RT = 32; };
template <> struct TrsvCfg<double> { static constexpr int RT = 16; };
constexpr int TS_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(TS_THREADS) lsolve_kernel(TrsvArgs a, const int* __restrict__ level_nodes,
                                                            const cx_t<T>* __restrict__ b, cx_t<T>* __restrict__ ynd,
                                                            cx_t<T>* __restrict__ u, const cx_t<T>* __restrict__ factor,
                                                            const int* __restrict__ active) {
  using C = cx_t<T>;
  constexpr int RT = TrsvCfg<T>::RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* y = reinterpret_cast<C*>(smem_raw);   // [ns][RT]
  const int node = level_nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int c0 = blockIdx.z * RT;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node], uoff = a.node_uoff[node];
  const C* f = factor + (size_t)p * a.factor_size;
  const C* Lss = f + a.node_fss[node];
  const C* Lbs = f + a.node_fbs[node];
  const int tid = threadIdx.x;
  // load b (natural order, gathered); i fastest for coalescing
  for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
    const int i = idx % ns, cc = idx / ns;
    const int c = c0 + cc;
    C v = mk<C>(0, 0);
    if (c < a.N) {
      const size_t s = (size_t)p * a.N + c;
      if (!active || active[s]) v = b[s * a.n + a.perm[off + i]];
    }
    y[i * RT + cc] = v;
  }
  __syncthreads();
  // subtract the descendants' update rows (cc fastest: u rows are [row][system])
  for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
    const int cc = idx % RT, i = idx / RT;
    const int c = c0 + cc;
    if (c >= a.N) continue;
    const size_t s = (size_t)p * a.N + c;
    C acc = y[i * RT + cc];
    const int e0 = a.contrib_ptr[off + i], e1 = a.contrib_ptr[off + i + 1];
    for (int e = e0; e < e1; ++e) acc = csub(acc, u[(size_t)a.contrib_idx[e] * a.S + s]);
    y[i * RT + cc] = acc;
  }
  __syncthreads();
  // unit lower triangular solve
  for (int k = 0; k < ns - 1; ++k) {
    const int rows = ns - k - 1;
    for (int idx = tid; idx < rows * RT; idx += TS_THREADS) {
      const int cc = idx % RT, i = k + 1 + idx / RT;
      y[i * RT + cc] = csub(y[i * RT + cc], cmul(Lss[(size_t)i * ns + k], y[k * RT + cc]));
    }
    __syncthreads();
  }
  // store y (ND order)
  for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
    const int i = idx % ns, cc = idx / ns;
    const int c = c0 + cc;
    if (c < a.N) ynd[((size_t)p * a.N + c) * a.n + off + i] = y[i * RT + cc];
  }
  // update rows u = L_BS y
  for (int idx = tid; idx < nb * RT; idx += TS_THREADS) {
    const int cc = idx % RT, j = idx / RT;
    const int c = c0 + cc;
    if (c >= a.N) continue;
    const C* lr = Lbs + (size_t)j * ns;
    C acc = mk<C>(0, 0);
    for (int i = 0; i < ns; ++i) acc = cfma(lr[i], y[i * RT + cc], acc);
    u[(size_t)(uoff + j) * a.S + (size_t)p * a.N + c] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(TS_THREADS) usolve_kernel(TrsvArgs a, const int* __restrict__ level_nodes,
                                                            const cx_t<T>* __restrict__ ynd, cx_t<T>* __restrict__ x,
                                                            const cx_t<T>* __restrict__ factor,
                                                            const int* __restrict__ active) {
  using C = cx_t<T>;
  constexpr int RT = TrsvCfg<T>::RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int node = level_nodes[blockIdx.x];
  const int p = blockIdx.y;
  const int c0 = blockIdx.z * RT;
  const int ns = a.node_ns[node], nb = a.node_nb[node], off = a.node_off[node], boff = a.node_boff[node];
  C* y = reinterpret_cast<C*>(smem_raw);   // [ns][RT]
  C* xb = y + (size_t)ns * RT;             // [nb][RT]
  const C* f = factor + (size_t)p * a.factor_size;
  const C* Uss = f + a.node_fss[node];
  const C* Usb = f + a.node_fsb[node];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
    const int i = idx % ns, cc = idx / ns;
    const int c = c0 + cc;
    y[i * RT + cc] = (c < a.N) ? ynd[((size_t)p * a.N + c) * a.n + off + i] : mk<C>(0, 0);
  }
  for (int idx = tid; idx < nb * RT; idx += TS_THREADS) {
    const int j = idx % nb, cc = idx / nb;
    const int c = c0 + cc;
    xb[j * RT + cc] = (c < a.N) ? x[((size_t)p * a.N + c) * a.n + a.bnat[boff + j]] : mk<C>(0, 0);
  }
  __syncthreads();
  if (nb > 0) {
    for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
      const int cc = idx % RT, i = idx / RT;
      const C* ur = Usb + (size_t)i * nb;
      C acc = y[i * RT + cc];
      for (int j = 0; j < nb; ++j) acc = csub(acc, cmul(ur[j], xb[j * RT + cc]));
      y[i * RT + cc] = acc;
    }
    __syncthreads();
  }
  // upper solve: at step k, x_k = d_k y_k is final; rows i < k subtract U_ik x_k
  for (int k = ns - 1; k > 0; --k) {
    const C dk = Uss[(size_t)k * ns + k];
    for (int idx = tid; idx < k * RT; idx += TS_THREADS) {
      const int cc = idx % RT, i = idx / RT;
      const C xk = cmul(dk, y[k * RT + cc]);
      y[i * RT + cc] = csub(y[i * RT + cc], cmul(Uss[(size_t)i * ns + k], xk));
    }
    __syncthreads();
  }
  for (int idx = tid; idx < ns * RT; idx += TS_THREADS) {
    const int i = idx % ns, cc = idx / ns;
    const int c = c0 + cc;
    if (c >= a.N) continue;
    const size_t s = (size_t)p * a.N + c;
    if (active && !active[s]) continue;
    x[s * a.n + a.perm[off + i]] = cmul(Uss[(size_t)i * ns + i], y[i * RT + cc]);
  }
}

size_t trsv_smem_bytes(bool dbl, int max_ns, int max_nb) {
  const int RT = dbl ? TrsvCfg<double>::RT : TrsvCfg<float>::RT;
  const size_t cs = dbl ? sizeof(double2) : sizeof(float2);
  return (size_t)(max_ns + max_nb) * RT * cs;
}

template <typename T>
static cudaError_t run_t(const TrsvArgs& a, const TrsvLevels& lv, int P, const void* b, void* ynd, void* u, void* x,
                         const void* factor, const int* active, size_t smem, cudaStream_t st) {
  constexpr int RT = TrsvCfg<T>::RT;
  // the opt-in shared-memory limit only ever grows (handles of different grids share the kernels)
  static size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(lsolve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(usolve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  const int tiles = (a.N + RT - 1) / RT;
  for (int h = 0; h < lv.nlevels; ++h) {
    dim3 grid(lv.count[h], P, tiles);
    lsolve_kernel<T><<<grid, TS_THREADS, smem, st>>>(a, lv.nodes + lv.start[h], (const cx_t<T>*)b, (cx_t<T>*)ynd,
                                                     (cx_t<T>*)u, (const cx_t<T>*)factor, active);
  }
  for (int h = lv.nlevels - 1; h >= 0; --h) {
    dim3 grid(lv.count[h], P, tiles);
    usolve_kernel<T><<<grid, TS_THREADS, smem, st>>>(a, lv.nodes + lv.start[h], (const cx_t<T>*)ynd, (cx_t<T>*)x,
                                                     (const cx_t<T>*)factor, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_spp_solve(bool dbl, const TrsvArgs& a, const TrsvLevels& lv, int P, const void* b, void* ynd,
                             void* u, void* x, const void* factor, const int* active, size_t smem, cudaStream_t st) {
  if (dbl) return run_t<double>(a, lv, P, b, ynd, u, x, factor, active, smem, st);
  return run_t<float>(a, lv, P, b, ynd, u, x, factor, active, smem, st);
}

}  // namespace omm
