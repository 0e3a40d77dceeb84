// Gram C = A^H B on the 5th-generation tensor cores (tcgen05, kind::tf32) with a
// three-term split for FP32-level accuracy (eq. omm and Sec. 2.1: the N x N overlap
// matrices X^*X, X^*HX and the line-search blocks reduce over the grid, K = n).
//
// Complex to real: with a column stored as interleaved (re, im) pairs, a real dot product
// of two columns over K = 2n gives Re(a^H b); with b~ = (im, -re) pairs it gives Im(a^H b).
// So one CTA tile computes [Re | Im] = A^T [B | B~] as a real 128 x 256 product.
// Split: x = hi + lo with hi = x rounded to TF32 (19 leading bits) and lo = x - hi;
// A^T B ~ Ahi^T Bhi + Ahi^T Blo + Alo^T Bhi (the dropped lo*lo term is ~2^-22 relative).
// Operands are staged by the CTA's threads into shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix), in two stages so that staging
// overlaps the MMAs of the previous chunk; one elected thread issues the MMAs into a
// 128 x 256 FP32 accumulator in tensor memory; tcgen05.commit signals the stage's
// mbarrier; the epilogue reads the accumulator with tcgen05.ld and writes FP32 split-K
// partials, summed in FP64 in a fixed order by a second kernel.  Every mbarrier wait is
// bounded: on timeout the kernel records an error code and stops issuing work.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace omm {

namespace {

constexpr int TM = 128;        // rows of C per CTA (columns of A)
constexpr int TNB = 128;       // columns of B per CTA (-> 256 accumulator columns: Re | Im)
constexpr int TN = 2 * TNB;
constexpr int KF = 32;         // floats of K per stage (16 complex)
constexpr int THREADS = 256;       // 8 warps stage operands; warps 0..3 read the accumulator
constexpr uint32_t TMEM_COLS = 256;

// bytes per operand tile (KF floats per row, 4 bytes)
constexpr int A_BYTES = TM * KF * 4;    // 16 KB
constexpr int B_BYTES = TN * KF * 4;    // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;     // hi / lo tiles of one chunk
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;          // two stages + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in a K-major no-swizzle tile with KF floats per row:
// core matrix (row / 8, k / 4) at ((row / 8) * (KF / 4) + k / 4) * 128, inside it
// (row % 8) * 16 + (k % 4) * 4.  K-adjacent core matrices are 128 B apart (LBO), 8-row
// groups (KF / 4) * 128 B apart (SBO).
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(((row >> 3) * (KF / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

constexpr uint32_t LBO = 128;
constexpr uint32_t SBO = (KF / 4) * 128;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
  // base offset 0, LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = TN, M = TM
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// wait on phase parity with a wall-clock bound (non-blocking test in a polling loop);
// returns false after ~200 ms
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 200000000ull) return false;
  }
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

}  // namespace

// part: [splits][na][2 * nb] floats (Re block then Im block per row of C)
// Two operand stages: while the tensor core consumes the hi / lo tiles of chunk c, the
// CTA's threads stage chunk c + 1 into the other buffers; a buffer is overwritten only
// after the mbarrier of its previous use (the tcgen05.commit of chunk c - 2) completed.
__global__ void __launch_bounds__(THREADS, 1) gram_tc_kernel(const float* __restrict__ A, int na,
                                                             const float* __restrict__ B, int nb, size_t n,
                                                             size_t kchunk, float* __restrict__ part,
                                                             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand region: stage b at base + b * STAGE_BYTES
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int i0 = blockIdx.x * TM;      // rows of C (columns of A)
  const int j0 = blockIdx.y * TNB;     // columns of B
  const size_t kb = (size_t)blockIdx.z * kchunk;                  // complex index range
  const size_t ke = (kb + kchunk < n) ? kb + kchunk : n;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();   // the .sync.aligned tcgen05 instructions need a converged warp
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  uint32_t phase[2] = {0u, 0u};   // parity of the next completion of each stage's mbarrier
  int pending[2] = {0, 0};        // a commit of the stage not yet waited for
  const size_t ldf = 2 * n;       // floats per column
  // per thread: EA float pairs of A and EB of B per chunk, loaded one chunk ahead into
  // registers (all independent loads in flight at once), split and stored when the stage
  // is free
  constexpr int EA = TM * (KF / 2) / THREADS, EB = TNB * (KF / 2) / THREADS;
  float2 va[EA], vb[EB];
  auto load_chunk = [&](size_t k0) {
#pragma unroll
    for (int q = 0; q < EA; ++q) {
      const int e = tid + q * THREADS;
      const int r = e / (KF / 2), pr = e % (KF / 2);
      const size_t kc = k0 + pr;   // complex index
      va[q] = (i0 + r < na && kc < ke) ? *reinterpret_cast<const float2*>(A + (size_t)(i0 + r) * ldf + 2 * kc)
                                       : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < EB; ++q) {
      const int e = tid + q * THREADS;
      const int r = e / (KF / 2), pr = e % (KF / 2);
      const size_t kc = k0 + pr;
      vb[q] = (j0 + r < nb && kc < ke) ? *reinterpret_cast<const float2*>(B + (size_t)(j0 + r) * ldf + 2 * kc)
                                       : make_float2(0.f, 0.f);
    }
  };
  if (kb < ke) load_chunk(kb);
  int c = 0;
  for (size_t k0 = kb; k0 < ke; k0 += KF / 2, ++c) {
    const int sb = c & 1;
    unsigned char* sAh = base + sb * STAGE_BYTES;
    unsigned char* sAl = sAh + A_BYTES;
    unsigned char* sBh = sAl + A_BYTES;
    unsigned char* sBl = sBh + B_BYTES;
    if (pending[sb]) {   // the MMAs of chunk c - 2 must be done with this stage
      if (mbar_wait(&bar[sb], phase[sb])) {
        phase[sb] ^= 1u;
        pending[sb] = 0;
      } else {           // stays pending: the drain below waits once more before dealloc
        if (tid == 0) atomicExch(err, 1);
        abort_sh = 1;
      }
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
      if (abort_sh) break;
    }
    // ---- split this chunk (A: TM columns x KF floats; B: TNB columns -> B and B~) into
    // hi / lo tiles of the free stage
#pragma unroll
    for (int q = 0; q < EA; ++q) {
      const int e = tid + q * THREADS;
      const int r = e / (KF / 2), pr = e % (KF / 2);
      const float2 v = va[q];
      const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
      const uint32_t o = tile_off(r, 2 * pr);
      *reinterpret_cast<float2*>(sAh + o) = make_float2(hx, hy);
      *reinterpret_cast<float2*>(sAl + o) = make_float2(v.x - hx, v.y - hy);
    }
#pragma unroll
    for (int q = 0; q < EB; ++q) {
      const int e = tid + q * THREADS;
      const int r = e / (KF / 2), pr = e % (KF / 2);
      const float2 v = vb[q];
      const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
      const uint32_t o = tile_off(r, 2 * pr);
      const uint32_t ot = tile_off(TNB + r, 2 * pr);
      *reinterpret_cast<float2*>(sBh + o) = make_float2(hx, hy);
      *reinterpret_cast<float2*>(sBl + o) = make_float2(v.x - hx, v.y - hy);
      // B~ = (im, -re)
      *reinterpret_cast<float2*>(sBh + ot) = make_float2(hy, -hx);
      *reinterpret_cast<float2*>(sBl + ot) = make_float2(v.y - hy, -(v.x - hx));
    }
    // the next chunk's loads are in flight while this chunk is issued and consumed
    if (k0 + KF / 2 < ke) load_chunk(k0 + KF / 2);
    // make the generic-proxy shared stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
      for (int s = 0; s < KF / 8; ++s) {   // K = 8 tf32 per MMA = 2 core matrices = 256 bytes
        const uint32_t off = s * 256;
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bh + off), (c == 0 && s == 0) ? 0u : 1u);
        mma_tf32(tmem, smem_desc(ah + off), smem_desc(bl + off), 1u);
        mma_tf32(tmem, smem_desc(al + off), smem_desc(bh + off), 1u);
      }
      mma_commit(&bar[sb]);
    }
    pending[sb] = 1;
  }
  // ---- the last (one or two) commits, and after a timeout the batch that did not
  // finish in time (bounded again), before the accumulator is read or freed
  for (int sb = 0; sb < 2; ++sb) {
    if (!pending[sb]) continue;
    if (!mbar_wait(&bar[sb], phase[sb])) {
      if (tid == 0) atomicExch(err, 1);
      abort_sh = 1;
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  // ---- epilogue (warps 0..3: TMEM lanes 32 w .. 32 w + 31 = rows of C; column = [Re | Im]
  // index).  The condition is uniform across each warp (tcgen05.ld is .sync.aligned).
  if (!abort_sh && kb < ke && warp < 4) {
    const int row = warp * 32 + lane;
    float* out = part + ((size_t)blockIdx.z * na + (i0 + row)) * (2 * (size_t)nb);
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      __syncwarp();
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i0 + row < na) {
        const int part_half = c0 / TNB;             // 0: Re, 1: Im
        const int jc = j0 + (c0 % TNB);
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (jc + q < nb) out[(size_t)part_half * nb + jc + q] = __uint_as_float(r[q]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

__global__ void gram_tc_reduce_kernel(const float* __restrict__ part, int ks, int na, int nb, double2* __restrict__ C,
                                      int ldc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= na * nb) return;
  const int i = idx / nb, j = idx % nb;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < ks; ++z) {
    const float* p = part + ((size_t)z * na + i) * (2 * (size_t)nb);
    re += (double)p[j];
    im += (double)p[nb + j];
  }
  C[(size_t)i * ldc + j] = make_double2(re, im);
}

namespace {
int tc_splits(int na, int nb, size_t n) {
  const int tiles = ((na + TM - 1) / TM) * ((nb + TNB - 1) / TNB);
  int ks = (152 + tiles - 1) / tiles;          // about one CTA per SM
  const int maxks = (int)((n + 511) / 512);
  if (ks > maxks) ks = maxks;
  return ks < 1 ? 1 : ks;
}
}  // namespace

size_t gram_tc_work_bytes(int na, int nb, size_t n) {
  return sizeof(float) * (size_t)tc_splits(na, nb, n) * na * 2 * nb + 256;
}

bool gram_tc_supported(size_t n) { return n % (KF / 2) == 0; }

cudaError_t launch_gram_tc(const void* A, int na, const void* B, int nb, size_t n, double2* C, int ldc, void* work,
                           int* err, cudaStream_t st) {
  if (na <= 0 || nb <= 0) return cudaSuccess;
  cudaError_t e0 = raise_smem_limit((const void*)gram_tc_kernel);
  if (e0 != cudaSuccess) return e0;
  int ks = tc_splits(na, nb, n);
  size_t kchunk = (n + ks - 1) / ks;
  kchunk = (kchunk + (KF / 2) - 1) / (KF / 2) * (KF / 2);
  ks = (int)((n + kchunk - 1) / kchunk);
  float* part = (float*)work;
  dim3 grid((na + TM - 1) / TM, (nb + TNB - 1) / TNB, ks);
  gram_tc_kernel<<<grid, THREADS, SMEM_BYTES, st>>>((const float*)A, na, (const float*)B, nb, n, kchunk, part, err);
  const int tot = na * nb;
  gram_tc_reduce_kernel<<<(tot + 255) / 256, 256, 0, st>>>(part, ks, na, nb, C, ldc);
  return cudaGetLastError();
}

}  // namespace omm
