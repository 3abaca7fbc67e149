// kf_tma.cuh -- Tensor Memory Accelerator (cp.async.bulk.tensor) loads into
// shared memory, completed through mbarriers, with bounded waits.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kf {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make mbarrier initialisation and prior generic shared-memory writes visible
// to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// try_wait with a suspend-time hint: a waiting warp is parked (up to ~1 us)
// instead of spinning, so co-resident warps keep the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
      : "memory");
  return done != 0;
}

// Wait for the phase `parity` of `bar` with at most `limit` polls (each may
// park the warp for up to the hint).  Returns false if the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// TMA destinations in shared memory are kept 128-byte aligned.
constexpr int TMA_SMEM_ALIGN = 128;

__device__ __forceinline__ float *align_smem(float *p) {
  return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(p) + TMA_SMEM_ALIGN - 1) &
                                   ~(uintptr_t)(TMA_SMEM_ALIGN - 1));
}

// 3-D tiled TMA load of one box at coordinates (x, y, z) into shared memory
// (destination 128-byte aligned); x times the element size (4 or 2 bytes)
// must be a multiple of 16.  A destination or coordinate that breaks these
// rules is not issued: the function returns false and the caller's bounded
// wait reports the failure.
__device__ __forceinline__ bool tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar, int elem_bytes = 4) {
  if ((smem_u32(dst) & (TMA_SMEM_ALIGN - 1)) != 0 || ((x * elem_bytes) & 15) != 0) return false;
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
  return true;
}

// 2-D tiled TMA load of one box at coordinates (x, y); the same rules.
__device__ __forceinline__ bool tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                            int elem_bytes = 4) {
  if ((smem_u32(dst) & (TMA_SMEM_ALIGN - 1)) != 0 || ((x * elem_bytes) & 15) != 0) return false;
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
  return true;
}

}  // namespace kf
