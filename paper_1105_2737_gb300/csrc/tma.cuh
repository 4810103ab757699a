// Helpers of the kernels that move data with the Tensor Memory Accelerator's
// bulk copies (cp.async.bulk): mbarrier set-up, bounded waits, loads from and
// stores to global memory.
#pragma once
#include "common.cuh"

namespace grf {
namespace tma {

constexpr unsigned kTmaSpinCap = 1u << 24;
constexpr unsigned long long kTmaTimeoutNs = 2000000000ull;  // 2 s

GRF_DEV unsigned long long tma_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

GRF_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

GRF_DEV void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// One bulk copy global -> shared of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completing `bytes` transactions on `bar`.
GRF_DEV void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Wait for the phase of `bar` with the given parity; false after the limits.
GRF_DEV bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (unsigned it = 0; it < kTmaSpinCap; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 0) {
      const unsigned long long t = tma_clock_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > kTmaTimeoutNs) return false;
    }
  }
  return false;
}

// One bulk copy shared -> global of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) in this thread's bulk group.  The generic-proxy writes to
// the source must be made visible to the async proxy first
// (fence.proxy.async.shared::cta, then a barrier if other threads wrote it).
GRF_DEV void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
GRF_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every bulk store this thread committed has read its source.
GRF_DEV void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
GRF_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tma
}  // namespace grf
