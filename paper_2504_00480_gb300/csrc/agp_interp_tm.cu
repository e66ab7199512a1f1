// Interpolation (NFFT, Appendix A) of d = 3 windows on the tensor cores, as a
// persistent, warp-specialised kernel with the A operand in tensor memory.
//
// The contraction is the one of agp_interp_tc.cu: for a run of up to four
// cells along the last dimension (one work unit of at most 256 points) and 16
// right-hand sides,
//     H[p, (u, r)] = sum_{(t1, t2)} A[p, (t1, t2)] B[(u, r), (t1, t2)],
//     A = psi1_p(t1) psi2_p(t2),   B = G[t1, t2, u][r]  (the run's grid block),
// with split-TF32 products (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi) and FP32
// accumulation; then h_p(r) = sum_t3 psi3_p(t3) H[p, (t3 + delta_p, r)] and
// Out[perm p][r] += scale h_p(r) with vector atomics.
//
// Design (one CTA per SM, 18 warps, all 512 tensor-memory columns):
//  * The unit's points form two M tiles of 128 (one tensor-memory lane per
//    point), and every chunk of the grid block (B, K = 8 grid rows) feeds the
//    MMAs of both tiles: the block is read from L2 once per 256 points.
//  * A lives in tensor memory: the thread of a lane holds psi1 and psi2 of
//    its points of both tiles in registers (prefetched into shared memory
//    with cp.async during the previous unit) and writes each chunk's
//    products (hi and lo) with tcgen05.st; the chunk loop is unrolled, so
//    every product's factors are fixed at compile time.
//  * Warps 10-17 read each chunk's grid values from L2 (two chunks ahead, in
//    registers) and store them split into hi and lo in shared memory; warp 1
//    issues the MMAs from one thread; warps 2-5 form A; warps 6-9 contract
//    finished accumulators with psi3 and add the results into the output.
//    The two tiles' accumulators (208 columns each) are drained one after
//    the other, each with its own mbarrier, so the next unit's MMAs on tile
//    0 start while tile 1 is still being read.
//  * Work items (unit, 16-column half) in a fixed stride; every wait is
//    bounded and watches the CTA's abort word (as in agp_spread_tm.cu).
#include <algorithm>
#include <type_traits>

#include "agp_nufft_kernels.cuh"
#include "agp_tm.cuh"

namespace agp {
namespace {

constexpr int kImKC = 8;                        // grid rows (t1, t2) per chunk (K)
constexpr int kImRH = 16;                       // right-hand sides per work item
constexpr int kImMP = 128;                      // points per M tile
constexpr int kImMT = kRunPoints / kImMP;       // M tiles per unit
constexpr int kImNB = 4;                        // B operand ring
constexpr int kImLBO = 128;
constexpr int kImSBO = (kImKC / 4) * 128;
constexpr int kImBG = 4;                        // groups of 64 B-forming threads
constexpr int kImWarps = 18;
constexpr int kImThreads = kImWarps * 32;
constexpr int kIWMma = 1, kIWA0 = 2, kIWE0 = 6, kIWB0 = 10;
constexpr int kImDCols = 208;                   // one tile's accumulator
constexpr int kImACol = kImMT * kImDCols;       // A buffers after the accumulators
constexpr int kImCols = 512;
static_assert(kImMT == 2, "two M tiles per unit");

template <int S>
struct ImShape {
  static constexpr int TT = 2 * S, TTP = ttp_of(S);
  static constexpr int ROWS = TT * TT;                          // K
  static constexpr int NCH = (ROWS + kImKC - 1) / kImKC;        // chunks per item
  static constexpr int T3M = TT + kRunCells - 1;
  static constexpr int NN = T3M * kImRH;
  static constexpr int NRG = NN / 8;                            // B row groups
  static constexpr int BPER = (NRG + kImBG - 1) / kImBG;        // row groups per B thread (max)
  static constexpr int WPP = wpp_of(3, S);
  static constexpr int PSI = 2 * TTP;                           // psi1, psi2 of a point as stored
  static constexpr int B_BYTES = NN * kImKC * 4;                // one of hi / lo
  static constexpr int OFF_P = kImNB * 2 * B_BYTES;             // A formers' prefetch slots
  // floats per point in a slot: both tiles' psi1, psi2, plus 4 of padding so
  // that the 16-byte reads of 8 consecutive lanes fall on distinct banks
  static constexpr int PST = kImMT * PSI + 4;
  static constexpr int SMEM = OFF_P + 2 * kImMP * PST * 4;
  static_assert(NN <= kImDCols, "tile shape");
  static_assert(kImACol + 2 * 32 <= kImCols, "tensor memory budget");
  static_assert(PSI % 4 == 0 && OFF_P % 16 == 0 && (PST / 4) % 2 == 1,
                "16-byte prefetch pieces, an odd number of them per point");
};

struct ImBars {
  uint64_t a_full[2], a_empty[2];
  uint64_t b_full[kImNB], b_empty[kImNB];
  uint64_t d_full, d_empty[kImMT];
  uint64_t drain;
};

template <int S>
__global__ void __launch_bounds__(kImThreads, 1)
k_interp_tm(const WinDev<float>* __restrict__ wins, int n_win, const int4* __restrict__ units,
            int64_t n_units, float* __restrict__ Out, int64_t ldo, int R, float scale, int rc,
            int* __restrict__ err, long long spin) {
  using Sh = ImShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, WPP = Sh::WPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ImBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  __shared__ WinDev<float> s_win[kMaxWindows];   // the plan's windows, read by every role
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nh = rc / kImRH;
  const int64_t n_items = n_units * nh;
  volatile int* abort = &abort_word;
  auto bbuf = [&](int b) { return reinterpret_cast<float*>(smem_raw + b * 2 * Sh::B_BYTES); };

  for (int q = tid; q < n_win; q += blockDim.x) s_win[q] = wins[q];
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.a_full[b], 4);
      mbar_init(&bars.a_empty[b], 1);
    }
    for (int b = 0; b < kImNB; ++b) {
      mbar_init(&bars.b_full[b], 8);
      mbar_init(&bars.b_empty[b], 1);
    }
    mbar_init(&bars.d_full, 1);
    for (int t = 0; t < kImMT; ++t) mbar_init(&bars.d_empty[t], 4);
    mbar_init(&bars.drain, 1);
    abort_word = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "n"(kImCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // work item i = (unit, half); every item holds points and columns (the
  // dispatcher requires R > rc - 16, and units are never empty)
  struct Item {
    int4 u;
    int r0, mt;       // first column, M tiles holding points
  };
  auto unit_at = [&](int64_t i) -> int4 {
    return i < n_items ? __ldg(units + (nh == 2 ? i >> 1 : i)) : make_int4(0, 0, 0, 0);
  };
  auto item_from = [&](int64_t i, int4 u, Item& it) {
    it.u = u;
    it.r0 = (nh == 2 ? (int)(i & 1) : 0) * kImRH;
    it.mt = u.w > kImMP ? 2 : 1;
  };

  if (warp == kIWMma) {
    // ---- MMA issue: the warp walks the items, lane 0 issues -------------------
    int64_t g = 0, nd = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);
      Item it;
      item_from(i, uc, it);
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
      const uint32_t idesc = umma_idesc_tf32(kImMP, nu * kImRH);
      bool ok = true;
      for (int c = 0; c < Sh::NCH; ++c, ++g) {
        const int ab = (int)(g & 1), bb = (int)(g % kImNB);
        // tile t's accumulator is free once the epilogue has read the previous
        // item's (waited before the item's first MMA on it)
        if (!warp_wait(&bars.a_full[ab], (uint32_t)((g >> 1) & 1), spin, abort) ||
            !warp_wait(&bars.b_full[bb], (uint32_t)((g / kImNB) & 1), spin, abort) ||
            (c == 0 && !warp_wait(&bars.d_empty[0], (uint32_t)((nd & 1) ^ 1), spin, abort))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const float* bh = bbuf(bb);
        const uint64_t dh = umma_desc(smem_u32(bh), kImLBO, kImSBO);
        const uint64_t dl = umma_desc(smem_u32(bh) + Sh::B_BYTES, kImLBO, kImSBO);
        const uint32_t a0 = tmem + (uint32_t)(kImACol + ab * 32);
        if (lane == 0) {
          mma_tf32_tmem_a(tmem, a0, dh, idesc, c > 0 ? 1u : 0u);
          mma_tf32_tmem_a(tmem, a0, dl, idesc, 1u);
          mma_tf32_tmem_a(tmem, a0 + 8, dh, idesc, 1u);
        }
        __syncwarp();
        if (c == 0 && !warp_wait(&bars.d_empty[1], (uint32_t)((nd & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        if (it.mt > 1) {
          tc_fence_after();
          if (lane == 0) {
            const uint32_t d1 = tmem + (uint32_t)kImDCols;
            mma_tf32_tmem_a(d1, a0 + 16, dh, idesc, c > 0 ? 1u : 0u);
            mma_tf32_tmem_a(d1, a0 + 16, dl, idesc, 1u);
            mma_tf32_tmem_a(d1, a0 + 24, dh, idesc, 1u);
          }
        }
        if (lane == 0) {
          mma_commit(&bars.a_empty[ab]);
          mma_commit(&bars.b_empty[bb]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&bars.d_full);
      __syncwarp();
      ++nd;
    }
  } else if (warp >= kIWA0 && warp < kIWA0 + 4) {
    // ---- A = psi1 psi2 into tensor memory, one point per lane and tile -------------
    const int qd = warp & 3;
    const int p = qd * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)kImACol;
    // this thread's two prefetch slots (alternate items): psi1, psi2 (as
    // stored) of its point in each tile
    float* slots = reinterpret_cast<float*>(smem_raw + Sh::OFF_P) + p * Sh::PST;
    auto slot_of = [&](int64_t j) { return slots + (j & 1) * (kImMP * Sh::PST); };
    auto prefetch = [&](const Item& it, float* slot) {
      const WinDev<float> w = s_win[it.u.x & 0xFFFF];
#pragma unroll
      for (int t = 0; t < kImMT; ++t) {
        const int pt = t * kImMP + p;
        const bool live = pt < it.u.w;
        const float* src = w.wts + (int64_t)(it.u.z + (live ? pt : 0)) * WPP;
#pragma unroll
        for (int q = 0; q < Sh::PSI / 4; ++q)
          cp_async16_zfill(slot + t * Sh::PSI + q * 4, src + q * 4, live ? 16 : 0);
      }
    };
    int64_t g = 0, j = 0;
    int4 un = unit_at(blockIdx.x);
    if (blockIdx.x < n_items) {
      Item first;
      item_from(blockIdx.x, un, first);
      prefetch(first, slot_of(0));
    }
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x, ++j) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);
      Item it;
      item_from(i, uc, it);
      cp_async_wait_all();                            // this item's values, staged earlier
      const float* slot = slot_of(j);
      float a[kImMT][TT], b[kImMT][TT];
#pragma unroll
      for (int t = 0; t < kImMT; ++t)
#pragma unroll
        for (int q4 = 0; q4 < Sh::PSI / 4; ++q4) {   // 16-byte shared-memory reads
          const float4 v = reinterpret_cast<const float4*>(slot + t * Sh::PSI)[q4];
          const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int q = 4 * q4 + c;
            if (q < TT) a[t][q] = e[c];
            else if (q >= TTP && q - TTP < TT) b[t][q - TTP] = e[c];
          }
        }
      if (i + gridDim.x < n_items) {                  // the next item's values, in flight
        Item nx;
        item_from(i + gridDim.x, un, nx);
        prefetch(nx, slot_of(j + 1));
      }
      bool ok = true;
#pragma unroll
      for (int c = 0; c < Sh::NCH; ++c) {
        const int ab = (int)((g + c) & 1);
        if (!warp_wait(&bars.a_empty[ab], (uint32_t)((((g + c) >> 1) & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        uint32_t hl[kImMT][2][kImKC];
#pragma unroll
        for (int t = 0; t < kImMT; ++t)
#pragma unroll
          for (int k = 0; k < kImKC; ++k) {
            const int kk = c * kImKC + k;                // grid row (t1, t2), a constant
            const float x = kk < Sh::ROWS ? a[t][kk / TT] * b[t][kk % TT] : 0.0f;
            const float h = tf32_round(x);
            hl[t][0][k] = __float_as_uint(h);
            hl[t][1][k] = __float_as_uint(x - h);
          }
        tc_fence_after();
        const uint32_t ta = tq + (uint32_t)(ab * 32);
        tmem_st8(ta, hl[0][0]);
        tmem_st8(ta + 8, hl[0][1]);
        tmem_st8(ta + 16, hl[1][0]);
        tmem_st8(ta + 24, hl[1][1]);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.a_full[ab]);
      }
      if (!ok) break;
      g += Sh::NCH;
    }
    cp_async_wait_all();
  } else if (warp >= kIWB0 && warp < kIWB0 + 8) {
    // ---- B = the run's grid block (hi and lo) into shared memory ----------------
    // The chunks of all items form one sequence g = 0, 1, 2, ...; two register
    // sets take the even and the odd chunks, so that the L2 loads of chunk
    // g + 2 are in flight while chunks g and g + 1 are stored. Thread slot:
    // row r8 and column k4 of the core matrices of column quad kq; group grp
    // (of kImBG) takes row groups [grp NRG / kImBG, (grp + 1) NRG / kImBG).
    const int bt = tid - kIWB0 * 32;
    const int kq = (bt >> 5) & 1, r8 = lane >> 2, k4 = lane & 3, grp = bt >> 6;
    const int kk4 = kq * 4 + k4;                      // grid row within the chunk
    const int o = kq * 32 + lane;
    const int rga = grp * Sh::NRG / kImBG, rgb = (grp + 1) * Sh::NRG / kImBG;
    constexpr int CORE = (kImKC / 4) * 32;
    struct BCur {
      int64_t i;            // work item (n_items: done)
      int c;                // chunk within the item
      int W, nu;
      const float* gp0;     // grid column r0 + r8 at the unit's first cell
      int4 un;              // the next item's unit, loaded ahead
    };
    auto benter = [&](BCur& b, int4 u) {
      b.un = unit_at(b.i + gridDim.x);
      if (b.i >= n_items) return;
      Item it;
      item_from(b.i, u, it);
      const WinDev<float> w = s_win[it.u.x & 0xFFFF];
      int cc[3];
      decode_cell<3>(it.u.y, w.N, cc);
      b.W = w.W;
      b.nu = TT + max(1, it.u.x >> 16) - 1;
      b.gp0 = w.grid + (((int64_t)cc[0] * w.W + cc[1]) * w.W + cc[2]) * rc + it.r0 + r8;
    };
    auto badv = [&](BCur& b) {
      if (++b.c < Sh::NCH) return;
      b.c = 0;
      b.i += gridDim.x;
      benter(b, b.un);
    };
    auto bload = [&](const BCur& b, float* gb) {
      if (b.i >= n_items) return;
      const int kk = b.c * kImKC + kk4;
      const bool krow = kk < Sh::ROWS;
      const int t1 = krow ? kk / TT : 0, t2 = krow ? kk - (kk / TT) * TT : 0;
      const float* gp = b.gp0 + ((int64_t)t1 * b.W + t2) * b.W * rc;
#pragma unroll
      for (int q = 0; q < Sh::BPER; ++q) {
        const int rg = rga + q;
        gb[q] = (krow && rg < rgb && rg < 2 * b.nu) ? __ldg(gp + (rg >> 1) * rc + (rg & 1) * 8)
                                                    : 0.0f;
      }
    };
    int64_t g = 0;
    auto step = [&](BCur& b, float* gb) -> bool {
      if (b.i >= n_items || warp_aborted(abort)) return false;
      const int bb = (int)(g % kImNB);
      if (!warp_wait(&bars.b_empty[bb], (uint32_t)(((g / kImNB) & 1) ^ 1), spin, abort))
        return false;
      float* bh = bbuf(bb);
      float* bl = bh + Sh::B_BYTES / 4;
#pragma unroll
      for (int q = 0; q < Sh::BPER; ++q) {
        const int rg = rga + q;
        if (rg < rgb) {
          const float x = gb[q];
          const float h = tf32_round(x);
          bh[rg * CORE + o] = h;
          bl[rg * CORE + o] = x - h;
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.b_full[bb]);
      ++g;
      badv(b);
      badv(b);
      bload(b, gb);
      return true;
    };
    BCur ca{blockIdx.x, 0, 0, 0, nullptr, make_int4(0, 0, 0, 0)};
    benter(ca, unit_at(blockIdx.x));
    BCur cb = ca;
    badv(cb);
    float ga[Sh::BPER], gb2[Sh::BPER];
    bload(ca, ga);
    bload(cb, gb2);
    while (step(ca, ga) && step(cb, gb2)) {
    }
  } else if (warp >= kIWE0 && warp < kIWE0 + 4) {
    // ---- epilogue: contract with psi3, scale, add into the output rows -----------
    const int qd = warp & 3;
    const bool vec = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(Out) & 15) == 0);
    int64_t nd = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);
      Item it;
      item_from(i, uc, it);
      const WinDev<float> w = s_win[it.u.x & 0xFFFF];
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
      // this thread's point of each tile: perm index, cell within the run, psi3
      int64_t pi[kImMT];
      int delta[kImMT];
      float p3[kImMT][TT];
#pragma unroll
      for (int t = 0; t < kImMT; ++t) {
        const int pt = t * kImMP + qd * 32 + lane;
        const bool live = pt < it.u.w;
        const int jj = it.u.z + (live ? pt : 0);
        delta[t] = 0;
#pragma unroll
        for (int q = 1; q < kRunCells; ++q)
          delta[t] += (q < L && jj >= __ldg(w.cell_start + it.u.y + q)) ? 1 : 0;
        const float* pw = w.wts + (int64_t)jj * WPP + 2 * TTP;
#pragma unroll
        for (int q = 0; q < TT; ++q) p3[t][q] = live ? __ldg(pw + 2 * q) : 0.0f;
        pi[t] = live ? (int64_t)__ldg(w.perm + jj) : -1;
      }
      if (!warp_wait(&bars.d_full, (uint32_t)(nd & 1), spin, abort)) break;
      tc_fence_after();
#pragma unroll
      for (int t = 0; t < kImMT; ++t) {
        float acc[kImRH];
#pragma unroll
        for (int q = 0; q < kImRH; ++q) acc[q] = 0.0f;
        if (t < it.mt) {
#pragma unroll 1
          for (int u = 0; u < nu; ++u) {
            uint32_t v[kImRH];
            tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(t * kImDCols + u * kImRH),
                      v);
            const int t3 = u - delta[t];
            float ps = 0.0f;
#pragma unroll
            for (int q = 0; q < TT; ++q) ps = (q == t3) ? p3[t][q] : ps;
#pragma unroll
            for (int q = 0; q < kImRH; ++q) acc[q] = fmaf(ps, __uint_as_float(v[q]), acc[q]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars.d_empty[t]);
        if (t < it.mt && pi[t] >= 0) {
          float* dst = Out + pi[t] * ldo + it.r0;
#pragma unroll
          for (int c4 = 0; c4 < kImRH; c4 += 4) {
            if (it.r0 + c4 >= R) break;
            const float4 val = make_float4(scale * acc[c4], scale * acc[c4 + 1],
                                           scale * acc[c4 + 2], scale * acc[c4 + 3]);
            if (vec && it.r0 + c4 + 4 <= R) {
              atomicAdd(reinterpret_cast<float4*>(dst + c4), val);
            } else {
              const float vv[4] = {val.x, val.y, val.z, val.w};
              for (int q = 0; q < 4 && it.r0 + c4 + q < R; ++q) atomicAdd(dst + c4 + q, vv[q]);
            }
          }
        }
      }
      ++nd;
    }
  }

  // ---- teardown ------------------------------------------------------------------
  __syncthreads();
  if (*abort) {
    if (warp == kIWMma && lane == 0) {
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
                 "n"(kImCols));
  }
}

template <int S>
cudaError_t interp_tm_s(const WinDev<float>* wins, int n_win, const int4* units, int64_t n_units, float* Out,
                        int64_t ldo, int R, float scale, int rc, int* err, long long spin,
                        cudaStream_t st) {
  using Sh = ImShape<S>;
  cudaError_t e = cudaFuncSetAttribute(k_interp_tm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Sh::SMEM);
  if (e != cudaSuccess) return e;
  if (n_units <= 0) return cudaSuccess;
  if (n_win < 1 || n_win > kMaxWindows) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t items = n_units * (rc / kImRH);
  const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
  k_interp_tm<S><<<grid, kImThreads, Sh::SMEM, st>>>(wins, n_win, units, n_units, Out, ldo, R, scale,
                                                     rc, err, spin);
  return cudaGetLastError();
}

}  // namespace

bool interp_tm_supported(int d, int s, int RC, int R) {
  // every 16-column half of the pass must hold columns (the B formers walk
  // every item)
  return d == 3 && (RC == 32 || RC == 16) && (s == 4 || s == 5) && R > RC - kImRH;
}

cudaError_t interp_units_tm(const WinDev<float>* wins, int n_win, const int4* units, int64_t n_units, int s,
                            float* Out, int64_t ldo, int R, float scale, int rc, int* err,
                            long long spin, cudaStream_t st) {
  switch (s) {
    case 4: return interp_tm_s<4>(wins, n_win, units, n_units, Out, ldo, R, scale, rc, err, spin, st);
    case 5: return interp_tm_s<5>(wins, n_win, units, n_units, Out, ldo, R, scale, rc, err, spin, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace agp
