// Spreading (adjoint NFFT, Appendix A) of d = 3 windows on the 5th-generation
// tensor cores. For one work item (the points of one grid cell) the update
// of the cell's (2s)^3 x R block of grid values is a dense contraction over
// the points j:
//     G[(t1, t2), (t3, r)] += sum_j A[(t1, t2), j] B[(t3, r), j],
//     A[(t1, t2), j] = psi1_j(t1) psi2_j(t2),  B[(t3, r), j] = psi3_j(t3) v_j(r),
// (for a run of cells, t3 counts the block's planes and B[(u, r), j] is
// psi3_j(u - delta_j) v_j(r), delta_j the cell of point j within the run),
// i.e. a [(2s)^2 x m] x [m x 2s R] matrix product per item (m <= item size).
// Each CTA takes one run of up to four cells along the last dimension (its
// (2s)^2 x (2s + L - 1) block) and 16 of the 32 right-hand sides: M = 128 rows
// ((2s)^2 = 100 or 64, zero padded), N = (2s + L - 1) x 16 columns,
// accumulated in tensor memory (TMEM) by tcgen05.mma kind::tf32 over chunks
// of 16 points (two K = 8 steps). FP32 accuracy from TF32 inputs by the split
// x = x_hi + x_lo (x_hi = x rounded to TF32, x_lo = the exact remainder, of
// which the tensor cores use the TF32 bits, ~2^-21 relative to x):
//     A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// whose dropped term A_lo B_lo is ~2^-22 relative; products of TF32 values
// are exact and the tensor cores accumulate in FP32.
//
// Pipeline (384 threads): the window values and V rows of later chunks are
// staged with cp.async (kTcStages - 1 chunks ahead, perm indices one chunk
// before that) while all threads form chunk c's four operand matrices in shared memory (K-major, no
// swizzle: 8 x 16-byte core matrices, leading byte offset 128, stride byte
// offset 512; each thread owns one element slot of every core matrix it
// writes, so its window values are loaded once per chunk); one barrier per
// chunk, after which thread 0 issues the chunk's six MMAs and commits them
// to the buffer's mbarrier while the next chunk is formed in the other
// buffer. The epilogue reads TMEM (warp w owns lanes 32 (w % 4) .. + 31 =
// rows), transposes each 32 x 16 tile through shared memory and adds the
// block into the window's grid with vector atomics, four lanes per row.
// Every mbarrier wait is bounded (the plan's wait limit) and its outcome is
// agreed by the CTA at the chunk's barrier: on expiry the CTA stops issuing
// MMAs, drains the committed ones, records a timeout in the plan's error
// word, skips the epilogue and releases its TMEM.
#include <type_traits>

#include "agp_nufft_kernels.cuh"
#include "agp_tc.cuh"

namespace agp {
namespace {

#ifndef AGP_TC_THREADS
#define AGP_TC_THREADS 384          // threads per CTA of k_spread_tc (128 .. 512)
#endif
constexpr int kTcThreads = AGP_TC_THREADS;
#ifndef AGP_TC_STAGES
#define AGP_TC_STAGES 2             // staging buffers of k_spread_tc (prefetch distance + 1)
#endif
constexpr int kTcStages = AGP_TC_STAGES;
constexpr int kTcKC = 16;       // points per chunk
constexpr int kTcRH = 16;       // right-hand sides per CTA
constexpr int kTcLBO = 128;     // bytes between core matrices along K
constexpr int kTcSBO = (kTcKC / 4) * 128;   // bytes between 8-row groups

template <int S>
struct TcSpreadShape {
  static constexpr int TT = 2 * S, TTP = ttp_of(S);
  static constexpr int ROWS = TT * TT;
  static constexpr int RG8 = (ROWS + 7) / 8;          // 8-row groups written per chunk
  static constexpr int MR = 128;
  static constexpr int T3M = TT + kRunCells - 1;              // t3 planes of a run's block
  static constexpr int NN = T3M * kTcRH;                       // largest MMA N
  static constexpr int WPP = wpp_of(3, S);
  // staging row strides (floats) of a point's window values and V row, chosen
  // so that the loads of the operand formation (4 points x 8 rows per warp
  // instruction) spread over the shared-memory banks: 40 (s = 4) is free of
  // conflicts, 56 (s = 5) takes 33 wavefronts where 26 loads need 26 (44: 38);
  // V rows at stride 24 are conflict-free
  static constexpr int WPS = S == 4 ? 40 : (S == 5 ? 56 : WPP);
  static constexpr int VS = 24;
  static constexpr int A_BYTES = MR * kTcKC * 4;
  static constexpr int B_BYTES = NN * kTcKC * 4;
  static constexpr int OPND = 2 * A_BYTES + 2 * B_BYTES;     // hi and lo of A and B
  static constexpr int STG_W = kTcKC * WPS;                   // floats
  static constexpr int STG = (STG_W + kTcKC * VS) * 4;        // bytes
  static constexpr int SMEM = 2 * OPND + kTcStages * STG;
  static constexpr int TMEM_COLS = NN <= 128 ? 128 : 256;
  static_assert(ROWS <= MR, "(2s)^2 rows must fit one M = 128 tile");
  static_assert(NN % 16 == 0 && NN <= 256, "N must be a multiple of 16, at most 256");
  static_assert((WPP * 4) % 16 == 0 && WPS % 4 == 0 && WPS >= WPP && VS % 4 == 0 && VS >= kTcRH,
                "window values and V rows must be 16-byte rows");
};

// Operand formation of one chunk for thread group G (of NG) of a CTA, in the
// thread's fixed element slot (row r8, point k4 of every core matrix of point
// quad kq; element offset (row group (KC/4) + kq) 32 + lane). Fully unrolled:
// every store offset is a constant relative to the thread's base pointer.
template <int S, int G, int NG>
__device__ __forceinline__ void form_a(const float* __restrict__ pw, bool live, int r8,
                                       float* __restrict__ ph, float* __restrict__ pl) {
  using Sh = TcSpreadShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP;
  constexpr int RGA = G * Sh::RG8 / NG, RGB = (G + 1) * Sh::RG8 / NG;
  int row = RGA * 8 + r8;
  int t1 = row / TT, t2 = row - t1 * TT;
#pragma unroll
  for (int rg = RGA; rg < RGB; ++rg) {
    const float x = (live && row < Sh::ROWS) ? pw[t1] * pw[TTP + t2] : 0.0f;
    const float h = tf32_round(x);
    ph[rg * (kTcKC / 4) * 32] = h;
    pl[rg * (kTcKC / 4) * 32] = x - h;
    row += 8;
    t2 += 8;
    if (t2 >= TT) {
      t2 -= TT;
      ++t1;
    }
  }
}

// B rows n = 8 rg + r8 = (u, r): plane u of the run's block (u = rg / 2,
// the point's tap t3 = u - delta for its cell offset delta in the run),
// r = 8 (rg % 2) + r8; thread group G of NG takes its share of the planes
// u < nu. (An A row group costs more than a B plane, but moving B planes
// between the groups to even out their instruction counts was slower.)
template <int S, int G, int NG>
__device__ __forceinline__ void form_b(const float* __restrict__ p3, bool live, int delta, int nu,
                                       float v0, float v1, float* __restrict__ ph,
                                       float* __restrict__ pl) {
  constexpr int TT = 2 * S, T3M = TT + kRunCells - 1;
  constexpr int T3A = G * T3M / NG, T3B = (G + 1) * T3M / NG;
#pragma unroll
  for (int u = T3A; u < T3B; ++u) {
    if (u >= nu) break;
    const int t3 = u - delta;
    const float p = (live && t3 >= 0 && t3 < TT) ? p3[2 * t3] : 0.0f;
    const float x0 = p * v0, x1 = p * v1;
    const float h0 = tf32_round(x0), h1 = tf32_round(x1);
    ph[(2 * u) * (kTcKC / 4) * 32] = h0;
    pl[(2 * u) * (kTcKC / 4) * 32] = x0 - h0;
    ph[(2 * u + 1) * (kTcKC / 4) * 32] = h1;
    pl[(2 * u + 1) * (kTcKC / 4) * 32] = x1 - h1;
  }
}

template <int S>
__global__ void __launch_bounds__(kTcThreads)
k_spread_tc(const WinDev<float>* __restrict__ wins, const WinIO<float>* __restrict__ io,
            const int4* __restrict__ items, const float* __restrict__ V, int64_t ldv, int R,
            int rc, int* __restrict__ err, long long spin) {
  using Sh = TcSpreadShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, WPP = Sh::WPP, WPS = Sh::WPS, VS = Sh::VS;
  constexpr int KC = kTcKC, RH = kTcRH;
  static_assert(kTcThreads % 128 == 0 && kTcThreads <= 512, "groups of 128 threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nh = rc / 16;                         // 16-column halves of the grid rows
  const int4 it = items[blockIdx.x / nh];
  const int r0 = (blockIdx.x % nh) * RH;          // right-hand sides r0 .. r0 + 15
  if (r0 >= R) return;                            // whole CTA: nothing to add
  const int win = it.x & 0xFFFF, L = max(1, it.x >> 16);   // window, cells in the run
  const int nu = TT + L - 1;                      // planes of the run's block
  const WinDev<float> w = wins[win];
  if (io) {
    V = io[win].V;
    ldv = io[win].ldv;
  }
  // first sorted point of cells 1 .. L-1 of the run: a point's cell offset
  // delta is the number of these it has reached
  int bnd[kRunCells - 1];
#pragma unroll
  for (int q = 0; q < kRunCells - 1; ++q)
    bnd[q] = (q + 1 < L) ? __ldg(w.cell_start + it.y + q + 1) : 0x7FFFFFFF;
  const bool vec_ok = (ldv % 4 == 0) && ((reinterpret_cast<uintptr_t>(V) & 15) == 0);
  const int j0 = it.z, m = it.w;
  // operand buffer b (0, 1) at smem_raw + b OPND; staging buffer q (0 .. kTcStages - 1)
  // at smem_raw + 2 OPND + q STG
  auto opnd = [&](int b) { return smem_raw + b * Sh::OPND; };
  auto stg = [&](int b) { return reinterpret_cast<float*>(smem_raw + 2 * Sh::OPND + b * Sh::STG); };

  // zero the padding rows of A (hi and lo) of both buffers once
  for (int b = 0; b < 2; ++b)
    for (int e = Sh::RG8 * 8 * KC + tid; e < Sh::MR * KC; e += kTcThreads) {
      reinterpret_cast<float*>(opnd(b))[e] = 0.0f;
      reinterpret_cast<float*>(opnd(b) + Sh::A_BYTES)[e] = 0.0f;
    }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "n"(Sh::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }

  // staging runs PD = kTcStages - 1 chunks ahead of the formation: thread
  // tid < 4 KC copies 16 bytes of one point's V row (point tid / 4, columns
  // r0 + 4 (tid % 4) ..), its perm index loaded one chunk before that; one
  // cp.async group is committed per chunk step (empty past the last chunk)
  constexpr int PD = kTcStages - 1;
  const int nchunk = (m + KC - 1) / KC;
  const int vq = tid >> 2, vk = (tid & 3) * 4;
  auto perm_of = [&](int c) -> int64_t {
    const int q = c * KC + vq;
    return (tid < 4 * KC && c < nchunk && q < m) ? (int64_t)__ldg(w.perm + j0 + q) : 0;
  };
  auto stage = [&](int c, int64_t pi) {
    if (c >= nchunk) {
      cp_async_commit();
      return;
    }
    float* sw = stg(c % kTcStages);
    float* sv = sw + Sh::STG_W;
    const int q0 = c * KC;
    const int ns = min(KC, m - q0);
    const float* wsrc = w.wts + (int64_t)(j0 + q0) * WPP;
    for (int e = tid; e < ns * (WPP / 4); e += kTcThreads) {
      const int q = e / (WPP / 4), c = e - q * (WPP / 4);     // point q, 16-byte chunk c
      cp_async16(sw + q * WPS + c * 4, wsrc + e * 4, 16);
    }
    if (vec_ok) {
      if (tid < 4 * KC && vq < ns) {
        const int valid = max(0, min(4, R - (r0 + vk)));
        cp_async16(sv + vq * VS + vk, V + pi * ldv + (valid > 0 ? r0 + vk : 0), valid * 4);
      }
    } else {
      for (int e = tid; e < ns * RH; e += kTcThreads) {
        const int q = e / RH, r = e % RH;
        const int64_t i = __ldg(w.perm + j0 + q0 + q);
        sv[q * VS + r] = (r0 + r < R) ? V[i * ldv + r0 + r] : 0.0f;
      }
    }
    cp_async_commit();
  };

  const uint32_t idesc = umma_idesc_tf32(Sh::MR, nu * RH);
  // this thread's slot in every core matrix it writes: row r8 and point k4
  // within the core, point quad kq, and its share g of the row groups
  const int slot = tid & 127, g = tid >> 7;
  const int kq = slot >> 5, r8 = (lane >> 2), k4 = lane & 3;
  const int kk = kq * 4 + k4;                      // point within the chunk
  bool ok = true;
  for (int c = 0; c < PD; ++c) stage(c, perm_of(c));
  int64_t pf = perm_of(PD);
  cp_async_wait<PD - 1>();                 // chunk 0 staged
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  int issued = 0;                          // chunks whose MMAs are committed
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    stage(c + PD, pf);                     // its buffer was last read by chunk c - 1
    pf = perm_of(c + PD + 1);
    if (c >= 2 && !mbar_wait(&bar[b], ((c - 2) >> 1) & 1, spin)) ok = false;   // MMAs of chunk c-2
    const float* sw = stg(c % kTcStages);
    const float* sv = sw + Sh::STG_W;
    const bool live = kk < min(KC, m - c * KC);
    float* ahi = reinterpret_cast<float*>(opnd(b));
    float* alo = reinterpret_cast<float*>(opnd(b) + Sh::A_BYTES);
    float* bhi = reinterpret_cast<float*>(opnd(b) + 2 * Sh::A_BYTES);
    float* blo = reinterpret_cast<float*>(opnd(b) + 2 * Sh::A_BYTES + Sh::B_BYTES);
    {
      const float* pw = sw + kk * WPS;
      const float v0 = live ? sv[kk * VS + r8] : 0.0f;
      const float v1 = live ? sv[kk * VS + 8 + r8] : 0.0f;
      const int jj = j0 + c * KC + kk;             // this point's sorted index
      int delta = 0;
#pragma unroll
      for (int q = 0; q < kRunCells - 1; ++q) delta += jj >= bnd[q];
      const int o = kq * 32 + lane;
      constexpr int NG = kTcThreads / 128;
      auto form = [&](auto gc) {
        constexpr int G = decltype(gc)::value;
        form_a<S, G, NG>(pw, live, r8, ahi + o, alo + o);
        form_b<S, G, NG>(pw + 2 * TTP, live, delta, nu, v0, v1, bhi + o, blo + o);
      };
      switch (g) {
        case 0: form(std::integral_constant<int, 0>()); break;
        case 1: if constexpr (NG > 1) form(std::integral_constant<int, 1>()); break;
        case 2: if constexpr (NG > 2) form(std::integral_constant<int, 2>()); break;
        case 3: if constexpr (NG > 3) form(std::integral_constant<int, 3>()); break;
      }
    }
    cp_async_wait<PD - 1>();              // chunk c + 1 staged (this thread's copies)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    // operands of chunk c and staging of c + 1 complete; the CTA agrees on
    // whether every wait so far succeeded (on failure: issue nothing more)
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // descriptors differ only in the start address field (address >> 4)
      const uint64_t a0 = umma_desc(smem_u32(ahi), kTcLBO, kTcSBO), a1 = umma_desc(smem_u32(alo), kTcLBO, kTcSBO);
      const uint64_t b0 = umma_desc(smem_u32(bhi), kTcLBO, kTcSBO), b1 = umma_desc(smem_u32(blo), kTcLBO, kTcSBO);
#pragma unroll
      for (int s2 = 0; s2 < KC / 8; ++s2) {
        const uint64_t off = (uint64_t)(s2 * 2 * kTcLBO) >> 4;
        mma_tf32(tmem, a0 + off, b0 + off, idesc, (c > 0 || s2 > 0) ? 1u : 0u);
        mma_tf32(tmem, a0 + off, b1 + off, idesc, 1u);
        mma_tf32(tmem, a1 + off, b0 + off, idesc, 1u);
      }
      mma_commit(&bar[b]);
    }
    issued = c + 1;
  }
  // The last commit covers every MMA of this CTA. Its barrier has no other
  // phase pending: the wait for the chunk two before it succeeded (else the
  // chunk would not have been issued).
  const int lc = issued - 1;
  const bool fin = issued == 0 || mbar_wait(&bar[lc & 1], (lc >> 1) & 1, spin);
  ok = __syncthreads_and(ok && fin);
  if (!ok && issued > 0) mbar_wait(&bar[lc & 1], (lc >> 1) & 1);   // drain before TMEM is freed
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows (t1, t2)); with more
    // than four warps the t3 range is split between the warps of a quarter.
    // Each 32 x 16 tile (rows x right-hand sides) goes through shared memory
    // (the operand buffers are free now) so that four lanes cover one row's
    // 16 contiguous values: every vector atomic instruction of a warp then
    // touches 8 rows x 64 bytes instead of 32 rows x 16 bytes. The tile's
    // rows are 16 floats; 16-byte chunk c of row l sits at chunk position
    // c ^ ((l >> 1) & 3), so that both the row-wise writes and the
    // four-lanes-per-row reads of 16-byte vectors are free of bank conflicts.
    constexpr int NQ = kTcThreads / 128;              // warps per lane quarter
    const int quarter = warp % 4, part = warp / 4;
    float* tile = reinterpret_cast<float*>(smem_raw) + warp * (32 * 16);
    int cc[3];
    decode_cell<3>(it.y, w.N, cc);
    const int ta = part * nu / NQ, tb = (part + 1) * nu / NQ;
    const int c4 = (lane & 3) * 4;
#pragma unroll 1
    for (int t3 = ta; t3 < tb; ++t3) {              // plane of the run's block
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t3 * RH);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
            "tcgen05.wait::ld.sync.aligned;"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(tile + lane * 16 + ((c ^ ((lane >> 1) & 3)) << 2)) =
            make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]),
                        __uint_as_float(v[4 * c + 2]), __uint_as_float(v[4 * c + 3]));
      __syncwarp();
#pragma unroll
      for (int q8 = 0; q8 < 4; ++q8) {
        const int rl = q8 * 8 + (lane >> 2);            // row within the quarter
        const int row = quarter * 32 + rl;
        if (row < Sh::ROWS && r0 + c4 < R) {
          const int t1 = row / TT, t2 = row - (row / TT) * TT;
          const int64_t base = ((int64_t)(cc[0] + t1) * w.W + (cc[1] + t2)) * w.W + cc[2] + t3;
          const float4 val = *reinterpret_cast<const float4*>(
              tile + rl * 16 + (((lane & 3) ^ ((rl >> 1) & 3)) << 2));
          atomicAdd(reinterpret_cast<float4*>(w.grid + base * rc + r0 + c4), val);
        }
      }
      __syncwarp();
    }
  } else if (tid == 0) {
    atomicOr(err, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(Sh::TMEM_COLS));
}

template <int S>
cudaError_t spread_tc_s(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                        int64_t n_items, const float* V, int64_t ldv, int R, int rc, int* err,
                        long long spin, cudaStream_t st) {
  using Sh = TcSpreadShape<S>;
  cudaError_t e = cudaFuncSetAttribute(k_spread_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Sh::SMEM);
  if (e != cudaSuccess) return e;
  if (n_items <= 0) return cudaSuccess;
  k_spread_tc<S><<<(unsigned)(rc / 16 * n_items), kTcThreads, Sh::SMEM, st>>>(
      wins, io, items, V, ldv, R, rc, err, spin);
  return cudaGetLastError();
}

}  // namespace

bool spread_tc_supported(int d, int s, int RC) {
  return d == 3 && (RC == 32 || RC == 16) && (s == 4 || s == 5);
}

cudaError_t spread_items_tc(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                            int64_t n_items, int s, const float* V, int64_t ldv, int R, int rc,
                            int* err, long long spin, cudaStream_t st) {
  switch (s) {
    case 4: return spread_tc_s<4>(wins, io, items, n_items, V, ldv, R, rc, err, spin, st);
    case 5: return spread_tc_s<5>(wins, io, items, n_items, V, ldv, R, rc, err, spin, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace agp
