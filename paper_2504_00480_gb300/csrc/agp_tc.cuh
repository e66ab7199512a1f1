// tcgen05 helpers shared by the tensor-core spreading and interpolation:
// shared-memory matrix and instruction descriptors (K-major operands without
// swizzle: 8-row x 16-byte core matrices), the TF32 hi/lo split, MMA issue
// and commit, and a bounded mbarrier wait.
//
// Wait discipline of the kernels that use them: every mbarrier wait polls at
// most `limit` times (the plan's wait limit, kTcSpinLimit by default); the
// outcome is agreed by the whole CTA at the next CTA barrier
// (__syncthreads_and), so every branch that follows -- MMA issue, TMEM loads,
// the epilogue -- is CTA-uniform. After a failed wait a CTA issues no further
// MMAs, drains the ones it committed with the fixed bound kTcSpinLimit,
// waits for its cp.async copies, sets the timeout bit in the error word,
// skips its epilogue and releases its TMEM.
#pragma once

#include <stdint.h>

namespace agp {
namespace {

constexpr long long kTcSpinLimit = 1ll << 26;
// Suspend-time hint of one try_wait poll (ns): a waiting thread sleeps until
// the phase completes or the hint runs out, instead of spinning on the issue
// slots that the working roles of the CTA need.
constexpr uint32_t kTcSuspendNs = 1000;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between
// core matrices along K, sbo = bytes between 8-row groups
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

// x rounded to the nearest TF32 value (10 fraction bits; ties away from zero)
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar))
               : "memory");
}

// bounded wait for the given phase parity (at most `limit` polls); false on
// expiry. The first poll is a non-blocking test, the later ones suspend the
// thread for up to kTcSuspendNs (try_wait), so a limit of 1 gives up at once
// unless the phase is already complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kTcSpinLimit) {
  const uint32_t a = smem_u32(bar);
  if (limit < 1) return false;
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(a), "r"(parity)
      : "memory");
  if (done) return true;
  for (long long it = 1; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace
}  // namespace agp
