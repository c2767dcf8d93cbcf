// Asynchronous-copy building blocks shared by the TMA-fed sweeps (tensor-core sweeps,
// stored-cost sweeps): mbarriers with bounded waits, 2-D tensor (TMA) loads, plain bulk
// copies and the generic/async proxy fence, as inline PTX for sm_103a.
//
// Every wait is bounded: after kWaitLimit polls, or kWaitNs nanoseconds of the global
// timer, the waiting thread records LAMP_E_TIMEOUT in the context's status word and sets
// the CTA's error flag, so that the other roles of the CTA stop issuing work and the
// kernel returns.  A poll that finds the phase incomplete suspends the thread for up to
// kSuspendNs (the try_wait time hint; the thread resumes when the phase completes), so
// waiting warps (the TMA producer and the MMA issuer, which wait most of the time) take
// few issue slots from the epilogue warps on their schedulers.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "lamp_common.cuh"

namespace lamp {
namespace async {

constexpr uint32_t kWaitLimit = 1u << 24;  // polls of a bounded mbarrier wait
constexpr int kTimeoutStatus = 6;          // LAMP_E_TIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (before the CTA barrier)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr uint32_t kSuspendNs = 20000;       // suspend-time hint of a waiting try_wait
constexpr uint64_t kWaitNs = 4000000000ull;  // a wait gives up after 4 s

__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// the global timer (nanoseconds)
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase of the given parity; false when the CTA's error flag is set
// or the limit ran out (then the flag and the context status are set)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, DevState* dev,
                                          uint32_t limit = kWaitLimit) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait_hint(bar, parity)) return true;
    if (*(volatile int*)err) return false;
    if (global_ns() - t0 > kWaitNs) break;
  }
  atomicExch(err, 1);
  atomicExch(&dev->status, kTimeoutStatus);
  return false;
}

// drain wait used on the error path: only the iteration limit, no early exit
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return;
}

// 2-D tiled TMA load of one box at coordinates (c0 innermost, c1); c0 times the element
// size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// plain (untiled) bulk copy global -> shared, completion counted on an mbarrier;
// both addresses 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// orders this thread's generic-proxy accesses of shared memory before later async-proxy
// accesses (bulk and tensor copies) that other threads issue after synchronising with it:
// a consumer that read a buffer issues it before releasing the buffer to the next copy
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace async
}  // namespace lamp
