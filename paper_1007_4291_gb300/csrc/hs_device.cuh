// Device helpers of libhs: 1D TMA bulk copies into shared memory completed on
// an mbarrier, bounded barrier waits, and the plan's device status word.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "hs_internal.cuh"

namespace hs {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive once on `bar` and announce `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory; completion is signalled on `bar`.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Plain arrive (no transaction bytes): consumer release of a ring stage.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of phase `parity` of `bar`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `budget` clock cycles,
// polling with the non-blocking probe (no suspension of the warp).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Per-thread asynchronous copies global -> shared (8 or 16 bytes, naturally
// aligned), grouped by commit; wait_group N returns once at most N of the
// thread's most recent groups are still in flight.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Record the first error of the plan: code, block, column.
__device__ __forceinline__ void set_status(int* status, int code, int block, int col) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = block;
    status[2] = col;
  }
}

template <typename R> struct Shfl;
template <> struct Shfl<float> {
  static __device__ __forceinline__ float get(float v, int src, int width = 32) {
    return __shfl_sync(0xffffffffu, v, src, width);
  }
  static __device__ __forceinline__ float xr(float v, int m, int width = 32) {
    return __shfl_xor_sync(0xffffffffu, v, m, width);
  }
};
template <> struct Shfl<double> {
  static __device__ __forceinline__ double get(double v, int src, int width = 32) {
    return __shfl_sync(0xffffffffu, v, src, width);
  }
  static __device__ __forceinline__ double xr(double v, int m, int width = 32) {
    return __shfl_xor_sync(0xffffffffu, v, m, width);
  }
};
template <typename R> __device__ __forceinline__ cplx<R> shfl_c(cplx<R> v, int src, int width = 32) {
  return cplx<R>{Shfl<R>::get(v.re, src, width), Shfl<R>::get(v.im, src, width)};
}
template <typename R> __device__ __forceinline__ cplx<R> shfl_xor_c(cplx<R> v, int m, int width = 32) {
  return cplx<R>{Shfl<R>::xr(v.re, m, width), Shfl<R>::xr(v.im, m, width)};
}

// Row stride (complex elements) of the factor payloads in global memory: W+2
// keeps every row 16-byte aligned (128-bit shared-memory loads) and the rows
// read by the T row-slices of the sweep in distinct banks.
__host__ __device__ __forceinline__ int payload_ld(int W) { return W + 2; }

// Number of complex elements of one column payload of a block's factor:
// G (W x (W+2)), V (d_out x (W+2)), c (W), rounded up to an even count so
// that every payload is a multiple of 16 bytes.
__host__ __device__ __forceinline__ long long payload_elems(int W, int d_out) {
  long long e = (long long)(W + d_out) * payload_ld(W) + W;
  return (e + 1) & ~1LL;
}
// Reduced-system factors per separator, each W x (W+2): Gamma, F, and (at the
// twist separator only) the bottom coupling F'.
__host__ __device__ __forceinline__ long long red_elems(int W) { return 3LL * W * payload_ld(W); }
// Twist separator of a chain of K separators: the top and bottom halves of the
// reduced system are eliminated toward it from both ends.
__host__ __device__ __forceinline__ int twist_index(int K) { return K / 2; }
// Corner blocks per interior chunk: G_r, W_l, W_r, each W x (W+1) (setup only).
__host__ __device__ __forceinline__ long long cor_elems(int W) { return 3LL * W * (W + 1); }

}  // namespace hs
