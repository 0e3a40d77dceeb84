// Shared device/host helpers for the OMM library (complex arithmetic, error plumbing).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

#include "omm.h"

namespace omm {

// Complex type of a working precision: float2 for the mixed form, double2 for FP64.
template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C, typename S> __host__ __device__ __forceinline__ C cscale(C a, S s) {
  return mk<C>(a.x * s, a.y * s);
}
// a + b * c (complex fused)
template <typename C> __host__ __device__ __forceinline__ C cfma(C b, C c, C a) {
  return mk<C>(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// a + conj(b) * c
template <typename C> __host__ __device__ __forceinline__ C cfmac(C b, C c, C a) {
  return mk<C>(fma(b.x, c.x, fma(b.y, c.y, a.x)), fma(b.x, c.y, fma(-b.y, c.x, a.y)));
}
// multiply by i * sgn (sgn = +1 or -1)
template <int SGN, typename C> __host__ __device__ __forceinline__ C cmuli(C a) {
  return SGN > 0 ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }

template <typename Cd, typename Cs> __host__ __device__ __forceinline__ Cd ccast(Cs a) {
  Cd r; r.x = (decltype(r.x))a.x; r.y = (decltype(r.y))a.y; return r;
}

// Raise a kernel's opt-in dynamic shared-memory limit to the most the device allows
// (given its static shared memory), once per kernel and thread-safely; the limit is a
// ceiling only, the launch's dynamic size still sets the occupancy.
cudaError_t raise_smem_limit(const void* func);

// Programmatic dependent launch.  A kernel launched with `overlap` set may be scheduled
// while the kernel before it on the stream is still running.  griddep_wait() returns once
// that kernel has completed and its writes are visible (at once for an ordinary launch);
// griddep_launch() lets the next such kernel be scheduled.  Before griddep_wait() a kernel
// only reads data that nothing in the chain writes (factor values, index lists) and writes
// nothing; it calls griddep_launch() after the wait, so at most two kernels of a chain are
// resident at a time and the second one only runs its prologue early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool overlap, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

}  // namespace omm

#define OMM_CUDA_TRY(expr)                                              \
  do {                                                                  \
    cudaError_t _e = (expr);                                            \
    if (_e != cudaSuccess) {                                            \
      omm_internal_set_cuda_error(_e, #expr, __FILE__, __LINE__);       \
      return OMM_ECUDA;                                                 \
    }                                                                   \
  } while (0)

#define OMM_TRY(expr)                      \
  do {                                     \
    omm_status _s = (expr);                \
    if (_s != OMM_OK) return _s;           \
  } while (0)

extern "C++" void omm_internal_set_cuda_error(cudaError_t e, const char* what, const char* file, int line);
