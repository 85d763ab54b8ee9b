// Tensor-memory-accelerator (TMA) tile loads with mbarrier completion, as inline PTX for sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hydot {

// Upper bound on polls of an mbarrier before a kernel gives up, flags HYDOT_ERR_TIMEOUT and
// returns (each poll may itself suspend for a hardware-defined interval).
constexpr uint32_t WAIT_POLLS = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}

// Makes the initialised barrier visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}

// One arrival (no transaction bytes) by the executing thread.
__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(m)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` with at most `limit` polls; false when the limit was reached.
__device__ __forceinline__ bool mbar_wait_polls(uint64_t* m, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

// Bounded wait used by the pipelined kernels.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* m, uint32_t parity) {
  return mbar_wait_polls(m, parity, WAIT_POLLS);
}

// 4-D tiled tensor load global -> shared; coordinates innermost first. The x coordinate times the
// element size must be a multiple of 16 bytes; out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* m, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(m))
      : "memory");
}

}  // namespace hydot
