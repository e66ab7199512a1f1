// Interpolation (NFFT, Appendix A) of d = 3 windows on the tensor cores, as a
// persistent, warp-specialised kernel with the A operand in tensor memory.
//
// The contraction is the one of agp_interp_tc.cu: for a run of up to four
// cells along the last dimension, a tile of up to 128 of its points and 16
// right-hand sides,
//     H[p, (u, r)] = sum_{(t1, t2)} A[p, (t1, t2)] B[(u, r), (t1, t2)],
//     A = psi1_p(t1) psi2_p(t2),   B = G[t1, t2, u][r]  (the run's grid block),
// M = 128 points, N = 16 (2s + L - 1), K = the (2s)^2 grid rows in chunks of
// 16, split-TF32 products (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi) with FP32
// accumulation; then h_p(r) = sum_t3 psi3_p(t3) H[p, (t3 + delta_p, r)] and
// Out[perm p][r] += scale h_p(r) with vector atomics.
//
// Design (one CTA per SM, 18 warps, all 512 tensor-memory columns):
//  * A lives in tensor memory, one point per lane: the thread of a lane
//    keeps its point's psi1 and psi2 in registers and writes each chunk's 16
//    products (hi and lo) with tcgen05.st.
//  * Warps 10-17 read each chunk's grid values from L2 (one chunk ahead, in
//    registers) and store them split into hi and lo in shared memory (B);
//    warp 1 issues the MMAs from one thread; warps 2-5 form A; warps 6-9
//    contract finished accumulators with psi3 and add the results into the
//    output. Two accumulators of 208 columns let the epilogue of one work
//    item overlap the main loop of the next; roles hand buffers over through
//    mbarriers only.
//  * Work items (tile of at most 128 points of one run, 16-column half) in a
//    fixed stride;
//    every wait is bounded and watches the CTA's abort word (as in
//    agp_spread_tm.cu).
#include <algorithm>
#include <type_traits>

#include "agp_nufft_kernels.cuh"
#include "agp_tm.cuh"

namespace agp {
namespace {

constexpr int kImKC = 16;                       // grid rows (t1, t2) per chunk (K)
constexpr int kImRH = 16;                       // right-hand sides per work item
constexpr int kImMP = kTilePoints;              // points per tile (M)
constexpr int kImNB = 3;                        // B operand ring
constexpr int kImLBO = 128;
constexpr int kImSBO = (kImKC / 4) * 128;
constexpr int kImWarps = 18;
constexpr int kImThreads = kImWarps * 32;
constexpr int kIWMma = 1, kIWA0 = 2, kIWE0 = 6, kIWB0 = 10;
constexpr int kImDCols = 208;
constexpr int kImACol = 2 * kImDCols;
constexpr int kImCols = 512;
static_assert(kImMP == 128, "one tensor-memory lane per point");

template <int S>
struct ImShape {
  static constexpr int TT = 2 * S, TTP = ttp_of(S);
  static constexpr int ROWS = TT * TT;                          // K
  static constexpr int NCH = (ROWS + kImKC - 1) / kImKC;        // chunks per item
  static constexpr int T3M = TT + kRunCells - 1;
  static constexpr int NN = T3M * kImRH;
  static constexpr int NRG = NN / 8;                            // B row groups
  static constexpr int BPER = NRG / 2;                          // row groups per B thread
  static constexpr int WPP = wpp_of(3, S);
  static constexpr int B_BYTES = NN * kImKC * 4;
  static constexpr int SMEM = kImNB * 2 * B_BYTES;
  static_assert(NN <= kImDCols && NRG % 2 == 0, "tile shape");
  static_assert(kImACol + 64 <= kImCols, "tensor memory budget");
};

struct ImBars {
  uint64_t a_full[2], a_empty[2];
  uint64_t b_full[kImNB], b_empty[kImNB];
  uint64_t d_full[2], d_empty[2];
  uint64_t drain;
};

template <int S>
__global__ void __launch_bounds__(kImThreads, 1)
k_interp_tm(const WinDev<float>* __restrict__ wins, const int4* __restrict__ units,
            int64_t n_units, float* __restrict__ Out, int64_t ldo, int R, float scale, int rc,
            int* __restrict__ err, long long spin) {
  using Sh = ImShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, WPP = Sh::WPP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ ImBars bars;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_word;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nh = rc / kImRH;
  const int64_t n_items = n_units * nh;
  volatile int* abort = &abort_word;
  auto bbuf = [&](int b) { return reinterpret_cast<float*>(smem_raw + b * 2 * Sh::B_BYTES); };

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.a_full[b], 4);
      mbar_init(&bars.a_empty[b], 1);
      mbar_init(&bars.d_full[b], 1);
      mbar_init(&bars.d_empty[b], 4);
    }
    for (int b = 0; b < kImNB; ++b) {
      mbar_init(&bars.b_full[b], 8);
      mbar_init(&bars.b_empty[b], 1);
    }
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

  // work item i = (tile, half): a tile is a run's unit of at most 128 points
  struct Item {
    int4 u;
    int p0, np, r0;
  };
  // the tile of work item i (loaded one item ahead by every role)
  auto unit_at = [&](int64_t i) -> int4 {
    return i < n_items ? __ldg(units + i / nh) : make_int4(0, 0, 0, 0);
  };
  auto item_from = [&](int64_t i, int4 u, Item& it) -> bool {
    it.u = u;
    it.p0 = 0;
    it.np = min(kImMP, it.u.w);
    it.r0 = (int)(i % nh) * kImRH;
    return it.r0 < R && it.np > 0;
  };

  if (warp == kIWMma) {
    // ---- MMA issue: the warp walks the items, lane 0 issues -------------------
    int64_t g = 0, nd = 0;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
      const int db = (int)(nd & 1);
      if (!warp_wait(&bars.d_empty[db], (uint32_t)(((nd >> 1) & 1) ^ 1), spin, abort)) break;
      const uint32_t idesc = umma_idesc_tf32(kImMP, nu * kImRH);
      const uint32_t dt = tmem + (uint32_t)(db * kImDCols);
      bool ok = true;
      for (int c = 0; c < Sh::NCH; ++c, ++g) {
        const int ab = (int)(g & 1), bb = (int)(g % kImNB);
        if (!warp_wait(&bars.a_full[ab], (uint32_t)((g >> 1) & 1), spin, abort) ||
            !warp_wait(&bars.b_full[bb], (uint32_t)((g / kImNB) & 1), spin, abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t a0 = tmem + (uint32_t)(kImACol + ab * 32);
          const float* bh = bbuf(bb);
          const uint64_t dh = umma_desc(smem_u32(bh), kImLBO, kImSBO);
          const uint64_t dl = umma_desc(smem_u32(bh) + Sh::B_BYTES, kImLBO, kImSBO);
#pragma unroll
          for (int s2 = 0; s2 < kImKC / 8; ++s2) {
            const uint64_t off = (uint64_t)(s2 * 2 * kImLBO) >> 4;
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
  } else if (warp >= kIWA0 && warp < kIWA0 + 4) {
    // ---- A = psi1 psi2 into tensor memory, one point (lane) per thread ---------
    // The thread's point keeps psi1, psi2 in registers; the chunk loop is
    // unrolled, so every product picks its two factors at compile time. The
    // next item's values are loaded when an item starts.
    const int qd = warp & 3;
    const int p = qd * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)kImACol;
    struct Psi {
      float a[TT], b[TT];
    };
    auto psi_load = [&](const Item& it, bool valid) -> Psi {
      const bool live = valid && p < it.np;
      const float* pw =
          wins[valid ? it.u.x & 0xFFFF : 0].wts + (live ? (int64_t)(it.u.z + it.p0 + p) * WPP : 0);
      Psi v;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        v.a[t] = live ? __ldg(pw + t) : 0.0f;
        v.b[t] = live ? __ldg(pw + TTP + t) : 0.0f;
      }
      return v;
    };
    int64_t g = 0, pre = -1;                          // pre: the item whose values are in nv
    Psi cv, nv;
    int4 un = unit_at(blockIdx.x);
    for (int64_t i = blockIdx.x; i < n_items && !warp_aborted(abort); i += gridDim.x) {
      const int4 uc = un;
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      if (pre != i) nv = psi_load(it, true);          // not prefetched: load now
      cv = nv;
      Item nx;
      const bool nvalid = item_from(i + gridDim.x, un, nx);
      nv = psi_load(nx, nvalid);                      // the next item's values, in flight
      pre = nvalid ? i + gridDim.x : -1;
      bool ok = true;
#pragma unroll
      for (int c = 0; c < Sh::NCH; ++c) {
        const int ab = (int)((g + c) & 1);
        if (!warp_wait(&bars.a_empty[ab], (uint32_t)((((g + c) >> 1) & 1) ^ 1), spin, abort)) {
          ok = false;
          break;
        }
        uint32_t hi[kImKC], lo[kImKC];
#pragma unroll
        for (int k = 0; k < kImKC; ++k) {
          const int kk = c * kImKC + k;                  // grid row (t1, t2), a constant
          const float x = kk < Sh::ROWS ? cv.a[kk / TT] * cv.b[kk % TT] : 0.0f;
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
        if (lane == 0) mbar_arrive(&bars.a_full[ab]);
      }
      if (!ok) break;
      g += Sh::NCH;
    }
  } else if (warp >= kIWB0 && warp < kIWB0 + 8) {
    // ---- B = the run's grid block (hi and lo) into shared memory ----------------
    // The chunks of all items form one sequence g = 0, 1, 2, ...; two register
    // sets take the even and the odd chunks, so that the L2 loads of chunk
    // g + 2 are in flight while chunks g and g + 1 are stored.
    const int bt = tid - kIWB0 * 32;
    const int kq = (bt >> 5) & 3, r8 = lane >> 2, k4 = lane & 3, grp = bt >> 7;
    const int kk4 = kq * 4 + k4;                      // grid row within the chunk
    const int o = kq * 32 + lane;
    constexpr int CORE = (kImKC / 4) * 32;
    struct BCur {
      int64_t i;            // work item (n_items: done)
      int c;                // chunk within the item
      int W, nu;
      const float* gp0;     // grid column r0 + r8 at the unit's first cell
      int4 un;              // the next item's tile, loaded ahead
    };
    // enter item b.i whose tile is u (every item is valid: tiles hold points
    // and both halves hold columns)
    auto benter = [&](BCur& b, int4 u) {
      b.un = unit_at(b.i + gridDim.x);
      if (b.i >= n_items) return;
      Item it;
      item_from(b.i, u, it);
      const WinDev<float> w = wins[it.u.x & 0xFFFF];
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
    // this thread's B elements of chunk b.c: grid row kk = c KC + kk4, row
    // groups rg = grp BPER + q: plane rg / 2, columns r0 + 8 (rg % 2) + r8
    auto bload = [&](const BCur& b, float* gb) {
      if (b.i >= n_items) return;
      const int kk = b.c * kImKC + kk4;
      const bool krow = kk < Sh::ROWS;
      const int t1 = krow ? kk / TT : 0, t2 = krow ? kk - (kk / TT) * TT : 0;
      const float* gp = b.gp0 + ((int64_t)t1 * b.W + t2) * b.W * rc;
#pragma unroll
      for (int q = 0; q < Sh::BPER; ++q) {
        const int rg = grp * Sh::BPER + q;
        gb[q] = (krow && rg < 2 * b.nu) ? __ldg(gp + (rg >> 1) * rc + (rg & 1) * 8) : 0.0f;
      }
    };
    int64_t g = 0;
    // store chunk `b` (values in gb), then move b two chunks on and load it
    auto step = [&](BCur& b, float* gb) -> bool {
      if (b.i >= n_items || warp_aborted(abort)) return false;
      const int bb = (int)(g % kImNB);
      if (!warp_wait(&bars.b_empty[bb], (uint32_t)(((g / kImNB) & 1) ^ 1), spin, abort))
        return false;
      float* bh = bbuf(bb);
      float* bl = bh + Sh::B_BYTES / 4;
#pragma unroll
      for (int q = 0; q < Sh::BPER; ++q) {
        const int rg = grp * Sh::BPER + q;
        const float x = gb[q];
        const float h = tf32_round(x);
        bh[rg * CORE + o] = h;
        bl[rg * CORE + o] = x - h;
      }
      asm volatile("fence.proxy.async.shared::cta;");
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
      un = unit_at(i + gridDim.x);               // next item, in flight
      Item it;
      if (!item_from(i, uc, it)) continue;
      const WinDev<float> w = wins[it.u.x & 0xFFFF];
      const int L = max(1, it.u.x >> 16), nu = TT + L - 1;
      const int p = qd * 32 + lane;
      const bool live = p < it.np;
      const int jj = it.u.z + it.p0 + (live ? p : 0);
      int delta = 0;
#pragma unroll
      for (int q = 1; q < kRunCells; ++q)
        delta += (q < L && jj >= __ldg(w.cell_start + it.u.y + q)) ? 1 : 0;
      float p3[TT];
      const float* pw = w.wts + (int64_t)jj * WPP + 2 * TTP;
#pragma unroll
      for (int t = 0; t < TT; ++t) p3[t] = live ? __ldg(pw + 2 * t) : 0.0f;
      const int64_t pi = live ? (int64_t)__ldg(w.perm + jj) : 0;
      const int db = (int)(nd & 1);
      if (!warp_wait(&bars.d_full[db], (uint32_t)((nd >> 1) & 1), spin, abort)) break;
      tc_fence_after();
      float acc[kImRH];
#pragma unroll
      for (int q = 0; q < kImRH; ++q) acc[q] = 0.0f;
#pragma unroll 1
      for (int u = 0; u < nu; ++u) {
        uint32_t v[kImRH];
        tmem_ld16(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(db * kImDCols + u * kImRH), v);
        tmem_wait_ld();
        const int t3 = u - delta;
        float ps = 0.0f;
#pragma unroll
        for (int t = 0; t < TT; ++t) ps = (t == t3) ? p3[t] : ps;
#pragma unroll
        for (int q = 0; q < kImRH; ++q) acc[q] = fmaf(ps, __uint_as_float(v[q]), acc[q]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars.d_empty[db]);
      ++nd;
      if (live) {
        float* dst = Out + pi * ldo + it.r0;
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
cudaError_t interp_tm_s(const WinDev<float>* wins, const int4* units, int64_t n_units, float* Out,
                        int64_t ldo, int R, float scale, int rc, int* err, long long spin,
                        cudaStream_t st) {
  using Sh = ImShape<S>;
  cudaError_t e = cudaFuncSetAttribute(k_interp_tm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Sh::SMEM);
  if (e != cudaSuccess) return e;
  if (n_units <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t items = n_units * (rc / kImRH);
  const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
  k_interp_tm<S><<<grid, kImThreads, Sh::SMEM, st>>>(wins, units, n_units, Out, ldo, R, scale,
                                                     rc, err, spin);
  return cudaGetLastError();
}

}  // namespace

bool interp_tm_supported(int d, int s, int RC, int R) {
  // every 16-column half of the pass must hold columns (the B formers walk
  // every item)
  return d == 3 && (RC == 32 || RC == 16) && (s == 4 || s == 5) && R > RC - kImRH;
}

cudaError_t interp_units_tm(const WinDev<float>* wins, const int4* units, int64_t n_units, int s,
                            float* Out, int64_t ldo, int R, float scale, int rc, int* err,
                            long long spin, cudaStream_t st) {
  switch (s) {
    case 4: return interp_tm_s<4>(wins, units, n_units, Out, ldo, R, scale, rc, err, spin, st);
    case 5: return interp_tm_s<5>(wins, units, n_units, Out, ldo, R, scale, rc, err, spin, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace agp
