// Tensor-memory-accelerator copies and mbarrier waits for the FFT passes (sm_103a).
#pragma once
#include <cuda.h>  // CUtensorMap (the type only)
#include <cuda_runtime.h>

namespace tmk {

namespace {

// Copies by the tensor memory accelerator (cp.async.bulk.tensor, cp.async.bulk) that
// complete on an mbarrier.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(mb))
      : "memory");
}
// Wait for phase `parity` of the barrier to complete: at most kSpin polls of about a
// microsecond each; on timeout the status word is flagged and the caller goes on (its
// results are then invalid, and the host reports the flag), so no wait can hang.
constexpr int kSpin = 1 << 20;
__device__ __forceinline__ void mbar_wait(unsigned long long* mb, unsigned parity, unsigned* status) {
  unsigned done = 0;
  for (int i = 0; i < kSpin && !done; i++) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mb)), "r"(parity), "r"(1000u)
        : "memory");
  }
  if (!done && status) atomicOr(status, 1u);
}

// The same wait with a caller-given bound (polls >= 1); true if the phase completed.
__device__ __forceinline__ bool mbar_wait_limit(unsigned long long* mb, unsigned parity, int polls, unsigned* status) {
  unsigned done = 0;
  for (int i = 0; i < polls && !done; i++) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mb)), "r"(parity), "r"(1000u)
        : "memory");
  }
  if (!done && status) atomicOr(status, 1u);
  return done != 0;
}

// Orders this thread's view of shared memory (including what other threads read before
// a barrier it passed) before its following copies into shared memory by the async proxy:
// needed before a TMA overwrites a buffer that threads read with ordinary loads.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Orders global memory written by ordinary stores (of earlier kernels, seen through the
// dependent-launch wait) before this thread's following TMA reads of it.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

// named barrier `id` over n threads (0 is __syncthreads)
__device__ __forceinline__ void bar_named(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

// contiguous bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mb))
               : "memory");
}

}  // namespace

}  // namespace tmk
