// Tensor-memory-accelerator (TMA) loads into shared memory, tracked by an
// mbarrier, with a bounded wait.
//
// One thread arms the barrier with the number of bytes the copies will
// deliver (expect_tx) and issues the 2D tiled copies
// (cp.async.bulk.tensor.2d, box given by the tensor map); the copies complete
// the barrier's current phase when all their bytes have landed.  Waiters poll
// the phase with mbarrier.try_wait.parity at most kTmaPolls times: a copy that
// never lands cannot hang the kernel, the wait reports failure instead and the
// caller records an error status for the host.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace sp {

constexpr unsigned kTmaPolls = 1u << 20;   // try_wait polls before a wait gives up (each polls for a while)
constexpr int kStatusTmaTimeout = 1;       // device status word: a TMA wait gave up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barrier visible to the asynchronous proxy (the TMA unit)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// true when the phase of parity `parity` completed within `polls` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned polls) {
  for (unsigned i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// order this thread's earlier generic-proxy accesses to shared memory before
// asynchronous-proxy writes to it (a TMA load into a buffer just read)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// box at element coordinates (x, y) of the tensor map into shared memory at
// dst; x times the element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace sp
