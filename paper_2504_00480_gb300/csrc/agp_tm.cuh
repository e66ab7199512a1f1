// Helpers of the warp-specialised tensor-core kernels (agp_spread_tm.cu):
// mbarrier arrive / bounded waits that also watch a CTA-wide abort word,
// cp.async copies whose completion arrives on an mbarrier, tensor-memory
// stores and loads, and tcgen05.mma with the A operand in tensor memory.
//
// Wait discipline: a role that waits polls its mbarrier at most `limit`
// times (the first poll a non-blocking test, the later ones suspend the
// thread for up to kTcSuspendNs, waking when the phase completes) and gives up early when another role has raised the
// CTA's abort word; a wait that runs out raises it. Every role then leaves
// its loop, so no thread of the CTA can be left waiting on a barrier that
// will never complete.
#pragma once

#include <stdint.h>

#include "agp_tc.cuh"

namespace agp {
namespace {

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(
      smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(kTcSuspendNs)
      : "memory");
  return done != 0;
}

// Wait for the phase of the given parity; false if the CTA aborts (the abort
// word is raised here when `limit` polls pass without completion).
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, uint32_t parity, long long limit,
                                                volatile int* abort) {
  if (mbar_test(bar, parity)) return true;
  for (long long it = 1; it < limit; ++it) {
    if (*abort) return false;
    if (mbar_try(bar, parity)) return true;
  }
  *abort = 1;
  return false;
}

// mbar_wait_abort for every lane of a warp, with one outcome for the warp
// (the tcgen05 loads and stores that follow need the whole warp)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, long long limit,
                                          volatile int* abort) {
  return __all_sync(0xFFFFFFFFu, mbar_wait_abort(bar, parity, limit, abort));
}

// true when the CTA's abort word is raised (one answer for the whole warp)
__device__ __forceinline__ bool warp_aborted(volatile int* abort) {
  return __any_sync(0xFFFFFFFFu, *abort != 0);
}

// Arrive on `bar` and raise its transaction count by `bytes` (the bulk
// copies that complete on it).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16)
// whose completion counts against `bar`'s transaction count.
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(smem)), "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The calling thread's earlier cp.async copies arrive on `bar` when complete
// (the arrival is counted in the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}

// generic-proxy shared-memory writes made visible to the async proxy (the
// tensor cores read the B operand through it)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Element-wise add of a shared-memory box into global memory through a 4-d
// tensor map (coordinates innermost first), as one bulk copy of this
// thread's bulk group; the adds are atomic per element.
__device__ __forceinline__ void bulk_reduce_add_4d(const void* map, uint32_t smem, int c0, int c1,
                                                   int c2, int c3) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.4d.global.shared::cta.add.bulk_group [%0, {%2, %3, %4, %5}], [%1];"
      ::"l"(map), "r"(smem), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until this thread's bulk copies have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Wait until this thread's bulk copies are complete (their global writes done).
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// 4-byte cp.async (zero-filled past src_bytes), for rows that are not 16-byte aligned
__device__ __forceinline__ void cp_async4_zfill(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// 16 consecutive tensor-memory columns of the warp's 32 lanes (one value per lane and column)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}

// 8 consecutive tensor-memory columns of the warp's 32 lanes
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}

// 16 consecutive tensor-memory columns of the warp's 32 lanes, waited for in
// the same statement (the registers are valid when it returns)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;");
}

// D (tensor memory) += A (tensor memory, M lanes x K = 8 columns) x B
// (shared-memory descriptor); acc = 0 overwrites D.
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t dtmem, uint32_t atmem, uint64_t b,
                                                uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
      "r"(atmem), "l"(b), "r"(idesc), "r"(acc));
}

}  // namespace
}  // namespace agp
