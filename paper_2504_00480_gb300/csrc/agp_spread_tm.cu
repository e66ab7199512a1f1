// Spreading (adjoint NFFT, Appendix A) of d = 3 windows on the tensor cores,
// as a persistent, warp-specialised kernel with the A operand in tensor
// memory.
//
// The contraction is the one of agp_spread_tc.cu: for a run of up to four
// cells along the last dimension (one work unit of at most 256 points) and 16
// right-hand sides,
//     G[(t1, t2), (u, r)] += sum_j A[(t1, t2), j] B[(u, r), j],
//     A = psi1_j(t1) psi2_j(t2),   B = psi3_j(u - delta_j) v_j(r),
// M = 128 rows ((2s)^2 used), N = 16 (2s + L - 1), K = the unit's points in
// chunks of 16, with FP32 accuracy from TF32 products of split operands
// (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation).
//
// Design (one CTA per SM, 22 warps, all 512 tensor-memory columns):
//  * A lives in tensor memory: each of its 128 rows is one lane, written by
//    the thread of that lane (tcgen05.st); the tensor cores read it there,
//    so shared memory carries only B. Two A buffers (hi and lo, 32 columns
//    each) and two accumulators of 208 columns, so that the epilogue of one
//    work item overlaps the main loop of the next.
//  * Roles: warp 0 stages each chunk's window values and V rows with
//    cp.async (completion arrives on the stage's mbarrier); warp 1 issues
//    the MMAs from one thread; warps 2-5 form A (one row per thread); warps
//    10-21 form B (hi and lo) in shared memory; warps 6-9 copy finished
//    accumulators into a shared-memory tile laid out as the unit's grid box,
//    which one bulk tensor reduction (cp.reduce.async.bulk.tensor, add) adds
//    into the grid, so the grid update costs the load/store unit only the
//    tile's stores. The roles hand buffers to each other through mbarriers
//    only -- there is no CTA-wide barrier in the loop.
//  * Work items (unit, 16-column half) are taken in a fixed stride
//    (blockIdx.x + k gridDim.x), so every role walks the same sequence.
//  * Every wait is bounded (the plan's wait limit) and watches the CTA's
//    abort word; on expiry all roles leave their loops, the MMA thread
//    drains what it issued, the CTA records AGP_TIMEOUT and frees its
//    tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "agp_nufft_kernels.cuh"
#include "agp_tm.cuh"

namespace agp {
namespace {

constexpr int kTmKC = 16;                       // points per chunk (K)
constexpr int kTmRH = 16;                       // right-hand sides per work item
constexpr int kTmNS = 4;                        // staging ring
constexpr int kTmNB = 3;                        // B operand ring
constexpr int kTmLBO = 128;                     // bytes between core matrices along K
constexpr int kTmSBO = (kTmKC / 4) * 128;       // bytes between 8-row groups
constexpr int kTmBG = 3;                        // groups of four B-forming warps
constexpr int kTmWarps = 10 + 4 * kTmBG;
constexpr int kTmThreads = kTmWarps * 32;
constexpr int kWLoad = 0, kWMma = 1, kWA0 = 2, kWE0 = 6, kWB0 = 10;   // first warp of each role
constexpr int kTmDCols = 208;                   // one accumulator: up to 13 planes x 16 columns
constexpr int kTmACol = 2 * kTmDCols;           // A buffers after the two accumulators
constexpr int kTmCols = 512;

template <int S>
struct TmShape {
  static constexpr int TT = 2 * S, TTP = ttp_of(S);
  static constexpr int ROWS = TT * TT;
  static constexpr int T3M = TT + kRunCells - 1;
  static constexpr int NN = T3M * kTmRH;
  static constexpr int WPP = wpp_of(3, S);
  // staged row stride (floats): the stored layout, so that one bulk copy
  // stages a chunk's window values (for s = 5 the four points a warp of B
  // formers reads fall on distinct banks)
  static constexpr int WPS = WPP;
  static constexpr int VS = 24;
  static constexpr int STG_W = kTmKC * WPS;                         // floats
  static constexpr int STG = STG_W + kTmKC * VS;                    // floats per stage
  static constexpr int B_BYTES = NN * kTmKC * 4;                    // one of hi / lo
  static constexpr int OFF_B = kTmNS * STG * 4;
  // epilogue tile: a unit's accumulator block as the grid box it adds into,
  // [t1][t2][u][16 right-hand sides] in 64-byte rows with the tensor map's
  // 64-byte swizzle; placed at the first 1024-byte boundary after OFF_E
  static constexpr int EP_BYTES = T3M * ROWS * kTmRH * 4;
  static constexpr int OFF_E = OFF_B + kTmNB * 2 * B_BYTES;
  static constexpr int SMEM = OFF_E + 1024 + EP_BYTES;
  static_assert(ROWS <= 128 && NN <= kTmDCols && NN % 16 == 0, "tile shape");
  static_assert(OFF_B % 128 == 0 && (2 * B_BYTES) % 128 == 0, "operand alignment");
  static_assert(kTmACol + 64 <= kTmCols, "tensor memory budget");
};

// B rows of a chunk for the thread's slot, as in agp_spread_tc.cu: row
// n = 8 rg + r8 = (u, r), u = rg / 2, r = 8 (rg % 2) + r8; group G of kTmBG
// takes its share of the planes u < nu.
template <int S, int G>
__device__ __forceinline__ void tm_form_b(const float* __restrict__ p3, bool live, int delta,
                                          int nu, float v0, float v1, float* __restrict__ ph,
                                          float* __restrict__ pl) {
  constexpr int TT = 2 * S, T3M = TT + kRunCells - 1;
  constexpr int T3A = G * T3M / kTmBG, T3B = (G + 1) * T3M / kTmBG;
  constexpr int CORE = (kTmKC / 4) * 32;
#pragma unroll
  for (int u = T3A; u < T3B; ++u) {
    if (u >= nu) break;
    const int t3 = u - delta;
    const float p = (live && t3 >= 0 && t3 < TT) ? p3[2 * t3] : 0.0f;
    const float x0 = p * v0, x1 = p * v1;
    const float h0 = tf32_round(x0), h1 = tf32_round(x1);
    ph[(2 * u) * CORE] = h0;
    pl[(2 * u) * CORE] = x0 - h0;
    ph[(2 * u + 1) * CORE] = h1;
    pl[(2 * u + 1) * CORE] = x1 - h1;
  }
}

struct TmBars {
  uint64_t st_full[kTmNS], st_empty[kTmNS];
  uint64_t a_full[2], a_empty[2];
  uint64_t b_full[kTmNB], b_empty[kTmNB];
  uint64_t d_full[2], d_empty[2];
  uint64_t e_full, e_empty;                     // epilogue tile written / read by the reduction
  uint64_t drain;
};

template <int S>
__global__ void __launch_bounds__(kTmThreads, 1)
k_spread_tm(const WinDev<float>* __restrict__ wins, const unsigned char* __restrict__ grid_maps,
            int n_win, const int4* __restrict__ units,
            int64_t n_units, const float* __restrict__ V, int64_t ldv, int vec, int R,
            int rc, int* __restrict__ err, long long spin) {
  using Sh = TmShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, WPP = Sh::WPP, WPS = Sh::WPS, VS = Sh::VS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TmBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  __shared__ WinDev<float> s_win[kMaxWindows];   // the plan's windows, read by every role
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nh = rc / kTmRH;
  const int64_t n_items = n_units * nh;
  volatile int* abort = &abort_word;
  auto stage = [&](int s) { return reinterpret_cast<float*>(smem_raw) + s * Sh::STG; };
  auto bbuf = [&](int b) {
    return reinterpret_cast<float*>(smem_raw + Sh::OFF_B + b * 2 * Sh::B_BYTES);
  };

  for (int q = tid; q < n_win; q += blockDim.x) s_win[q] = wins[q];
  if (tid == 0) {
    for (int s = 0; s < kTmNS; ++s) {
      mbar_init(&bars.st_full[s], 1 + 32);             // bulk bytes + one cp.async arrival per lane
      mbar_init(&bars.st_empty[s], 4 + 4 * kTmBG);     // A and B forming warps
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.a_full[b], 4);
      mbar_init(&bars.a_empty[b], 1);                  // tcgen05.commit
      mbar_init(&bars.d_full[b], 1);
      mbar_init(&bars.d_empty[b], 4);
    }
    for (int b = 0; b < kTmNB; ++b) {
      mbar_init(&bars.b_full[b], 4 * kTmBG);
      mbar_init(&bars.b_empty[b], 1);
    }
    mbar_init(&bars.e_full, 4);
    mbar_init(&bars.e_empty, 1);
    mbar_init(&bars.drain, 1);
    abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "n"(kTmCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // the work items every role walks: (unit, half) with points and columns
  struct Item {
    int4 u;
    int r0, nchunk;
  };
  // the unit of work item i (loaded one item ahead by every role)
  auto unit_at = [&](int64_t i) -> int4 {
    return i < n_items ? __ldg(units + (nh == 2 ? i >> 1 : i)) : make_int4(0, 0, 0, 0);
  };
  auto item_from = [&](int64_t i, int4 u, Item& it) -> bool {
    it.u = u;
    it.r0 = (nh == 2 ? (int)(i & 1) : 0) * kTmRH;
    it.nchunk = (it.u.w + kTmKC - 1) / kTmKC;
    return it.r0 < R && it.u.w > 0;
  };

  if (warp == kWLoad) {
    // ---- staging: window values and V rows of every chunk -------------------
    // Lane l copies V pieces l and l + 32 of a chunk (points l / 4 and
    // 8 + l / 4 of the chunk). The perm indices of a whole unit (at most 256
    // points) sit in registers, lane l holding points l + 32 q; those of the
    // next unit are loaded when a unit starts, so no copy waits for a load.
    constexpr int PQ = kRunPoints / 32;
    struct Perms {
      int32_t v[PQ];
    };
    auto perms = [&](const Item& it, bool valid) -> Perms {
      const int32_t* pp = s_win[valid ? it.u.x & 0xFFFF : 0].perm + (valid ? it.u.z : 0);
      const int m = valid ? it.u.w : 0;
      Perms pr;
#pragma unroll
      for (int q = 0; q < PQ; ++q) {
        const int pt = q * 32 + lane;
        pr.v[q] = pt < m ? __ldg(pp + pt) : 0;
      }
      return pr;
    };
    Perms pc, pn;
    int64_t g = 0, pre = -1;                          // pre: the item whose indices are in pn
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);
      Item it;
      if (!item_from(i, uc, it)) continue;
      if (pre != i) pn = perms(it, true);            // not prefetched: load now
      pc = pn;
      Item nx;
      const bool nv = item_from(i + gridDim.x, un, nx);
      pn = perms(nx, nv);                             // the next item's indices, in flight
      pre = nv ? i + gridDim.x : -1;
      const WinDev<float> w = s_win[it.u.x & 0xFFFF];
      bool ok = true;
      for (int c = 0; c < it.nchunk; ++c, ++g) {
        const int s = (int)(g % kTmNS);
        if (!warp_wait(&bars.st_empty[s], (uint32_t)(((g / kTmNS) & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        float* sw = stage(s);
        float* sv = sw + Sh::STG_W;
        const int q0 = c * kTmKC, ns = min(kTmKC, it.u.w - q0);
        // points c KC + q sit in slot c / 2 of lane (c % 2) 16 + q
        int32_t slot = pc.v[0];
#pragma unroll
        for (int q = 1; q < PQ; ++q) slot = (q == (c >> 1)) ? pc.v[q] : slot;
        // window values: one bulk copy of the chunk's contiguous rows
        if (lane == 0) {
          mbar_arrive_expect_tx(&bars.st_full[s], (uint32_t)(ns * WPP * 4));
          bulk_g2s(sw, w.wts + (int64_t)(it.u.z + q0) * WPP, (uint32_t)(ns * WPP * 4),
                   &bars.st_full[s]);
        }
        // V rows: lane l copies 16-byte pieces of points l / 4 and 8 + l / 4
        // (zero beyond R); its copies arrive on the stage when complete
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = h * 8 + (lane >> 2), vk = (lane & 3) * 4;
          const int64_t pi = __shfl_sync(0xFFFFFFFFu, slot, (c & 1) * 16 + q);
          if (q < ns) {
            const int valid = max(0, min(4, R - (it.r0 + vk)));
            if (vec) {
              cp_async16_zfill(sv + q * VS + vk, V + pi * ldv + (valid > 0 ? it.r0 + vk : 0),
                               valid * 4);
            } else {                                   // rows not 16-byte aligned
#pragma unroll
              for (int e = 0; e < 4; ++e)
                cp_async4_zfill(sv + q * VS + vk + e,
                                V + pi * ldv + (e < valid ? it.r0 + vk + e : 0), e < valid ? 4 : 0);
            }
          }
        }
        cp_async_arrive(&bars.st_full[s]);
      }
      if (!ok) break;
    }
    // the bulk copies of the last stages may still be landing (after an
    // abort): wait for every issued stage's bytes before the CTA can leave
    for (int64_t gg = g > kTmNS ? g - kTmNS : 0; gg < g; ++gg)
      mbar_wait(&bars.st_full[gg % kTmNS], (uint32_t)((gg / kTmNS) & 1));
    cp_async_wait_all();
  } else if (warp == kWMma) {
    // ---- MMA issue: the warp walks the items, lane 0 issues -------------------
    {
      int64_t g = 0, nd = 0;
      int4 un = unit_at(blockIdx.x);
      for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
        const int4 uc = un;
        un = unit_at(i + gridDim.x);               // next item, in flight
        Item it;
        if (!item_from(i, uc, it)) continue;
        const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
        const int db = (int)(nd & 1);
        if (!warp_wait(&bars.d_empty[db], (uint32_t)(((nd >> 1) & 1) ^ 1), spin, abort))
          break;
        const uint32_t idesc = umma_idesc_tf32(128, nu * kTmRH);
        const uint32_t dt = tmem + (uint32_t)(db * kTmDCols);
        bool ok = true;
        for (int c = 0; c < it.nchunk; ++c, ++g) {
          const int ab = (int)(g & 1), bb = (int)(g % kTmNB);
          if (!warp_wait(&bars.a_full[ab], (uint32_t)((g >> 1) & 1), spin, abort) ||
              !warp_wait(&bars.b_full[bb], (uint32_t)((g / kTmNB) & 1), spin, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t a0 = tmem + (uint32_t)(kTmACol + ab * 32);
            const float* bh = bbuf(bb);
            const uint64_t dh = umma_desc(smem_u32(bh), kTmLBO, kTmSBO);
            const uint64_t dl = umma_desc(smem_u32(bh) + Sh::B_BYTES, kTmLBO, kTmSBO);
#pragma unroll
            for (int s2 = 0; s2 < kTmKC / 8; ++s2) {
              const uint64_t off = (uint64_t)(s2 * 2 * kTmLBO) >> 4;
              const uint32_t ah = a0 + (uint32_t)(s2 * 8), al = ah + 16;
              mma_tf32_tmem_a(dt, ah, dh + off, idesc, (c > 0 || s2 > 0) ? 1u : 0u);
              mma_tf32_tmem_a(dt, ah, dl + off, idesc, 1u);
              mma_tf32_tmem_a(dt, al, dh + off, idesc, 1u);
            }
            mma_commit(&bars.a_empty[ab]);
            mma_commit(&bars.b_empty[bb]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) mma_commit(&bars.d_full[db]);
        __syncwarp();
        ++nd;
      }
    }
  } else if (warp >= kWA0 && warp < kWA0 + 4) {
    // ---- A = psi1 psi2 into tensor memory, one row (lane) per thread -----------
    const int qd = warp & 3;                          // lane quarter this warp may access
    const int row = qd * 32 + lane;
    const bool vrow = row < Sh::ROWS;
    const int t1 = vrow ? row / TT : 0, t2 = vrow ? row - (row / TT) * TT : 0;
    const uint32_t tq = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)kTmACol;
    int64_t g = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      bool ok = true;
      for (int c = 0; c < it.nchunk; ++c, ++g) {
        const int s = (int)(g % kTmNS), ab = (int)(g & 1);
        if (!warp_wait(&bars.st_full[s], (uint32_t)((g / kTmNS) & 1), spin, abort) ||
            !warp_wait(&bars.a_empty[ab], (uint32_t)(((g >> 1) & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        const int ns = min(kTmKC, it.u.w - c * kTmKC);
        const float* sw = stage(s);
        uint32_t hi[kTmKC], lo[kTmKC];
#pragma unroll
        for (int k = 0; k < kTmKC; ++k) {
          const float x = (vrow && k < ns) ? sw[k * WPS + t1] * sw[k * WPS + TTP + t2] : 0.0f;
          const float h = tf32_round(x);
          hi[k] = __float_as_uint(h);
          lo[k] = __float_as_uint(x - h);
        }
        tc_fence_after();
        tmem_st16(tq + (uint32_t)(ab * 32), hi);
        tmem_st16(tq + (uint32_t)(ab * 32 + 16), lo);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bars.a_full[ab]);
          mbar_arrive(&bars.st_empty[s]);
        }
      }
      if (!ok) break;
    }
  } else if (warp >= kWB0 && warp < kWB0 + 4 * kTmBG) {
    // ---- B = psi3 v (hi and lo) into shared memory -------------------------------
    const int bt = tid - kWB0 * 32;
    const int slot = bt & 127, grp = bt >> 7;
    const int kq = slot >> 5, r8 = lane >> 2, k4 = lane & 3;
    const int kk = kq * 4 + k4;                       // point within the chunk
    const int o = kq * 32 + lane;
    struct Bnd {
      int v[kRunCells - 1];
    };
    auto bounds = [&](const Item& it, bool valid) -> Bnd {
      const int L = valid ? max(1, it.u.x >> 16) : 1;
      const int32_t* cs = s_win[valid ? it.u.x & 0xFFFF : 0].cell_start + (valid ? it.u.y : 0);
      Bnd b;
#pragma unroll
      for (int q = 0; q < kRunCells - 1; ++q) b.v[q] = (q + 1 < L) ? __ldg(cs + q + 1) : 0x7FFFFFFF;
      return b;
    };
    Bnd nb;
    int64_t pre = -1;
    int64_t g = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
      // first sorted point of cells 1 .. L-1 of the run (this item's, loaded
      // one item ahead)
      if (pre != i) nb = bounds(it, true);
      const Bnd bnd = nb;
      Item nx;
      const bool nvalid = item_from(i + gridDim.x, un, nx);
      nb = bounds(nx, nvalid);
      pre = nvalid ? i + gridDim.x : -1;
      bool ok = true;
      for (int c = 0; c < it.nchunk; ++c, ++g) {
        const int s = (int)(g % kTmNS), bb = (int)(g % kTmNB);
        if (!warp_wait(&bars.st_full[s], (uint32_t)((g / kTmNS) & 1), spin, abort) ||
            !warp_wait(&bars.b_empty[bb], (uint32_t)(((g / kTmNB) & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        const float* sw = stage(s);
        const float* sv = sw + Sh::STG_W;
        const bool live = kk < min(kTmKC, it.u.w - c * kTmKC);
        const float* pw = sw + kk * WPS;
        const float v0 = live ? sv[kk * VS + r8] : 0.0f;
        const float v1 = live ? sv[kk * VS + 8 + r8] : 0.0f;
        const int jj = it.u.z + c * kTmKC + kk;
        int delta = 0;
#pragma unroll
        for (int q = 0; q < kRunCells - 1; ++q) delta += jj >= bnd.v[q];
        float* bh = bbuf(bb);
        float* bl = bh + Sh::B_BYTES / 4;
        if (grp == 0)
          tm_form_b<S, 0>(pw + 2 * TTP, live, delta, nu, v0, v1, bh + o, bl + o);
        else if (grp == 1)
          tm_form_b<S, 1>(pw + 2 * TTP, live, delta, nu, v0, v1, bh + o, bl + o);
        else
          tm_form_b<S, 2>(pw + 2 * TTP, live, delta, nu, v0, v1, bh + o, bl + o);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bars.b_full[bb]);
          mbar_arrive(&bars.st_empty[s]);
        }
      }
      if (!ok) break;
    }
  } else if (warp >= kWE0 && warp < kWE0 + 4) {
    // ---- epilogue: accumulator -> shared tile -> one bulk tensor add into the grid ----
    // Each warp copies its 32 accumulator rows (t1, t2), one 16-column plane
    // u at a time, into the tile at their place in the unit's grid box
    // [t1][t2][u][r]; planes u >= nu are written as zeros. When all four
    // warps are done, lane 0 of the first adds the whole box into the grid
    // with one bulk reduction and waits until it has read the tile before
    // the tile is written again.
    const int qd = warp & 3;
    const int row = qd * 32 + lane;
    const bool wrow = row < Sh::ROWS;
    const bool wwarp = qd * 32 < Sh::ROWS;             // the warp holds rows of the block
    const uint32_t sbase = smem_u32(smem_raw);
    const uint32_t toff = ((sbase + (uint32_t)Sh::OFF_E + 1023u) & ~1023u) - sbase;
    unsigned char* tile = smem_raw + toff;
    const bool issuer = warp == kWE0;
    int64_t nd = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      const int db = (int)(nd & 1);
      if (!warp_wait(&bars.d_full[db], (uint32_t)((nd >> 1) & 1), spin, abort) ||
          !warp_wait(&bars.e_empty, (uint32_t)((nd & 1) ^ 1), spin, abort))
        break;
      tc_fence_after();
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
#pragma unroll 1
      for (int u = 0; u < Sh::T3M; ++u) {
        uint32_t v[16];
        if (wwarp && u < nu) {
          tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(db * kTmDCols + u * kTmRH), v);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = 0u;
        }
        if (wrow) {
          // 16-byte chunk c of the row: logical offset (row T3M + u) 64 + 16 c,
          // address bits 4-5 XOR bits 7-8 (64-byte swizzle; the tile is
          // 1024-byte aligned); eight consecutive rows fall on distinct banks
          const uint32_t l0 = (uint32_t)(row * Sh::T3M + u) * 64u;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t lo = l0 + (uint32_t)c * 16u;
            *reinterpret_cast<float4*>(tile + (lo ^ (((lo >> 7) & 3u) << 4))) =
                make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]),
                            __uint_as_float(v[4 * c + 2]), __uint_as_float(v[4 * c + 3]));
          }
        }
      }
      // the accumulator is read: back to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.d_empty[db]);
      // the tile's writes are ordered before the bulk copy engine reads it
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.e_full);
      if (issuer) {
        if (!warp_wait(&bars.e_full, (uint32_t)(nd & 1), spin, abort)) break;
        if (lane == 0) {
          const int win = it.u.x & 0xFFFF;
          int cc[3];
          decode_cell<3>(it.u.y, s_win[win].N, cc);
          bulk_reduce_add_4d(grid_maps + (size_t)win * kGridMapBytes, smem_u32(tile), it.r0,
                             cc[2], cc[1], cc[0]);
          bulk_wait_read();
          mbar_arrive(&bars.e_empty);
        }
        __syncwarp();
      }
      ++nd;
    }
    // the last reductions' global adds are done before the CTA leaves
    if (issuer && lane == 0) bulk_wait_all();
  }

  // ---- teardown ------------------------------------------------------------------
  __syncthreads();
  if (*abort) {
    if (warp == kWMma && lane == 0) {
      // every MMA this thread issued completes before the commit arrives
      mma_commit(&bars.drain);
      mbar_wait(&bars.drain, 0u);
    }
    if (tid == 0) atomicOr(err, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(kTmCols));
  }
}

template <int S>
cudaError_t spread_tm_s(const WinDev<float>* wins, const void* grid_maps, int n_win,
                        const int4* units, int64_t n_units, const float* V, int64_t ldv, int R,
                        int rc, int* err, long long spin, cudaStream_t st) {
  using Sh = TmShape<S>;
  cudaError_t e = cudaFuncSetAttribute(k_spread_tm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Sh::SMEM);
  if (e != cudaSuccess) return e;
  if (n_units <= 0) return cudaSuccess;
  if (n_win < 1 || n_win > kMaxWindows || grid_maps == nullptr) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t items = n_units * (rc / kTmRH);
  const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
  const int vec = (ldv % 4 == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0) ? 1 : 0;
  k_spread_tm<S><<<grid, kTmThreads, Sh::SMEM, st>>>(
      wins, static_cast<const unsigned char*>(grid_maps), n_win, units, n_units, V, ldv, vec, R, rc,
      err, spin);
  return cudaGetLastError();
}

}  // namespace

bool spread_tm_supported(int d, int s, int RC) {
  return d == 3 && (RC == 32 || RC == 16) && (s == 4 || s == 5);
}

cudaError_t spread_units_tm(const WinDev<float>* wins, const void* grid_maps, int n_win,
                            const int4* units, int64_t n_units, int s, const float* V,
                            int64_t ldv, int R, int rc, int* err, long long spin,
                            cudaStream_t st) {
  switch (s) {
    case 4:
      return spread_tm_s<4>(wins, grid_maps, n_win, units, n_units, V, ldv, R, rc, err, spin, st);
    case 5:
      return spread_tm_s<5>(wins, grid_maps, n_win, units, n_units, V, ldv, R, rc, err, spin, st);
  }
  return cudaErrorInvalidValue;
}

// The driver's tensor-map encoder, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

bool encode_grid_maps(const WinDev<float>* wins_host, const int* win_d, int n_win, int s,
                      void* out) {
  static_assert(sizeof(CUtensorMap) == kGridMapBytes, "tensor map size");
  if ((reinterpret_cast<uintptr_t>(out) & 63) != 0 || n_win < 1 || (s != 4 && s != 5))
    return false;
  unsigned char* o = static_cast<unsigned char*>(out);
  std::memset(o, 0, (size_t)2 * n_win * kGridMapBytes);
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (encode == nullptr) return false;
  const cuuint32_t tt = (cuuint32_t)(2 * s), t3m = (cuuint32_t)(2 * s + kRunCells - 1);
  for (int h = 0; h < 2; ++h) {
    const cuuint64_t rc = h ? 32 : 16;
    for (int q = 0; q < n_win; ++q) {
      if (win_d[q] != 3) continue;
      const WinDev<float>& w = wins_host[q];
      // grid element (r, a3, a2, a1) at ((a1 W + a2) W + a3) rc + r
      const cuuint64_t W = (cuuint64_t)w.W;
      const cuuint64_t dims[4] = {rc, W, W, W};
      const cuuint64_t strides[3] = {rc * 4, W * rc * 4, W * W * rc * 4};
      const cuuint32_t box[4] = {(cuuint32_t)kTmRH, t3m, tt, tt};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      CUtensorMap* m = reinterpret_cast<CUtensorMap*>(o + ((size_t)h * n_win + q) * kGridMapBytes);
      if (encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, w.grid, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
        return false;
    }
  }
  return true;
}

}  // namespace agp
