// mbarrier and TMA (cp.async.bulk.tensor) helpers for the staged collision
// sweeps, with bounded waits. Internal to libkbe (CUDA, sm_103a).
//
// Every wait on an mbarrier is bounded by one second of device time
// (%globaltimer) and a round count: a copy that never lands makes the caller
// flag kDevTimeout and stop instead of hanging the GPU.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "kbe_internal.cuh"

namespace kbe {

// cuTensorMapEncodeTiled from the driver (no link against libcuda), resolved
// once per process; NULL when the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kMbarWaitNs = 1000000000ull;   // one second per wait

// true when the phase with this parity has completed; false after one second
// of device time (%globaltimer) or `limit` rounds, whichever comes first
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int limit) {
  const unsigned a = smem_addr(bar);
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < limit; ++it) {
    if ((it & 255) == 255 && global_ns() - t0 > kMbarWaitNs) return false;
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, int x, int y, int z, int w,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}

constexpr int kMbarWaitLimit = 1 << 30;   // try_wait rounds (a backstop; the time limit comes first)

}  // namespace

}  // namespace kbe
