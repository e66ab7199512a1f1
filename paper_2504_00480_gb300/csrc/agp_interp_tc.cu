// Interpolation (NFFT, Appendix A) of d = 3 windows on the 5th-generation
// tensor cores. For the points of one work item (one grid cell) the first
// two dimensions of the separable window sum are a dense product over the
// (2s)^2 grid rows (t1, t2) of the cell's block:
//     H[p, (t3, r)] = sum_{(t1, t2)} A[p, (t1, t2)] B[(t3, r), (t1, t2)],
//     A[p, (t1, t2)] = psi1_p(t1) psi2_p(t2),  B[(t3, r), (t1, t2)] = G[t1, t2, t3][r],
// and the last dimension is contracted in the epilogue:
//     h_p(r) = sum_t3 psi3_p(t3) H[p, (t3 + delta_p, r)],
// delta_p the cell of point p within the run.
// Each CTA takes one run of up to four cells along the last dimension (tiles
// of up to 128 points, M = 128; the run's block has 2s + L - 1 planes t3) and
// 16 of the 32 right-hand sides (N = (2s + L - 1) x 16), accumulates H in TMEM with
// tcgen05.mma kind::tf32 over chunks of 16 grid rows (two K = 8 steps), with operands
// split into TF32 hi and lo parts (A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi),
// then contracts with psi3, and adds scale * h into the caller's output rows
// with vector atomics (other windows add into the same rows).
//
// Pipeline (256 threads): the tile's window values and perm indices are
// staged once; per chunk of 16 grid rows all threads form A (from the window
// values) and B (grid values read from L2, prefetched a chunk ahead into
// registers) in one of two operand buffers, and after one barrier thread 0
// issues the chunk's six MMAs (two K = 8 steps) and commits them to the
// buffer's mbarrier. Every mbarrier wait is bounded (the plan's wait limit)
// and its outcome agreed by the CTA at the next barrier: on expiry the CTA
// stops issuing MMAs, drains the committed ones, records a timeout in the
// plan's error word, skips its remaining epilogues and releases its TMEM.
#include <type_traits>

#include "agp_nufft_kernels.cuh"
#include "agp_tc.cuh"

namespace agp {
namespace {

constexpr int kItThreads = 256;
constexpr int kItKC = 16;                     // grid rows (t1, t2) per chunk
constexpr int kItRH = 16;                     // right-hand sides per CTA
constexpr int kItMP = 128;                    // points per tile
constexpr int kItLBO = 128;
constexpr int kItSBO = (kItKC / 4) * 128;
constexpr int kItNG = kItThreads / 128;       // formation groups (128 element slots each)

template <int S>
struct TcInterpShape {
  static constexpr int TT = 2 * S, TTP = ttp_of(S);
  static constexpr int ROWS = TT * TT;                       // K (grid rows)
  static constexpr int NCH = (ROWS + kItKC - 1) / kItKC;     // chunks per tile
  static constexpr int T3M = TT + kRunCells - 1;             // planes of a run's block
  static constexpr int NN = T3M * kItRH;                     // largest MMA N
  static constexpr int WPP = wpp_of(3, S);
  static constexpr int A_BYTES = kItMP * kItKC * 4;
  static constexpr int B_BYTES = NN * kItKC * 4;
  static constexpr int OPND = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int WS_BYTES = kItMP * WPP * 4;
  static constexpr int PB_BYTES = 2 * kItMP * 17 * 4;        // epilogue partial sums
  static constexpr int SMEM_USED =
      (2 * OPND > PB_BYTES ? 2 * OPND : PB_BYTES) + WS_BYTES + 2 * kItMP * 4;
  // at least 76 KB so that at most two CTAs (2 x 256 TMEM columns) share an SM
  static constexpr int SMEM = SMEM_USED > 76 * 1024 ? SMEM_USED : 76 * 1024;
  static constexpr int TMEM_COLS = NN <= 128 ? 128 : 256;
  static constexpr int BPER = NN / 8 / kItNG;                 // B row groups per thread
  static_assert((NN / 8) % kItNG == 0 && 16 % kItNG == 0, "row groups split evenly");
  static_assert(NN % 16 == 0 && NN <= 256, "N must be a multiple of 16, at most 256");
  static_assert((WPP * 4) % 16 == 0, "window values must be 16-byte rows");
};

// Operand formation for thread group G: the thread's element slot is row r8
// and column k4 of every core matrix of column quad kq; rows of group G are
// row groups [G * 16/NG, (G+1) * 16/NG) of A (points) and
// [G * NN/8/NG, (G+1) * NN/8/NG) of B ((t3, r)). Offsets relative to the
// thread's base pointers are compile-time constants.
template <int S, int G>
__device__ __forceinline__ void it_load_b(const float* __restrict__ gp, bool krow, int nrg, int rc,
                                          float* gb) {
  constexpr int NRG = (2 * S + kRunCells - 1) * kItRH / 8, PER = NRG / kItNG, RGA = G * PER;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int rg = RGA + q;             // plane rg / 2 (cell stride rc), columns 8 (rg % 2) ..
    gb[q] = (krow && rg < nrg) ? __ldg(gp + (rg >> 1) * rc + (rg & 1) * 8) : 0.0f;
  }
}

template <int S, int G>
__device__ __forceinline__ void it_store_b(const float* gb, float* __restrict__ bh,
                                           float* __restrict__ bl) {
  constexpr int NRG = (2 * S + kRunCells - 1) * kItRH / 8, PER = NRG / kItNG, RGA = G * PER;
  constexpr int CORE = (kItKC / 4) * 32;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const float x = gb[q];
    const float h = tf32_round(x);
    bh[(RGA + q) * CORE] = h;
    bl[(RGA + q) * CORE] = x - h;          // the tensor cores use its TF32 bits
  }
}

template <int S, int G>
__device__ __forceinline__ void it_form_a(const float* __restrict__ w1, const float* __restrict__ w2,
                                          int np, int r8, bool krow, float* __restrict__ ah,
                                          float* __restrict__ al) {
  constexpr int WPP = wpp_of(3, S), PER = 16 / kItNG, RGA = G * PER;
  constexpr int CORE = (kItKC / 4) * 32;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int rg = RGA + q;
    const int p = rg * 8 + r8;
    const float x = (krow && p < np) ? w1[rg * 8 * WPP] * w2[rg * 8 * WPP] : 0.0f;
    const float h = tf32_round(x);
    ah[rg * CORE] = h;
    al[rg * CORE] = x - h;
  }
}

template <int S>
__global__ void __launch_bounds__(kItThreads, 2)
k_interp_tc(const WinDev<float>* __restrict__ wins, const WinIO<float>* __restrict__ io,
            const int4* __restrict__ items, float* __restrict__ Out, int64_t ldo, int R,
            float scale, int rc, int* __restrict__ err, long long spin) {
  using Sh = TcInterpShape<S>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, WPP = Sh::WPP, KC = kItKC, RH = kItRH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nh = rc / 16;                         // 16-column halves of the grid rows
  const int4 it = items[blockIdx.x / nh];
  const int r0 = (blockIdx.x % nh) * RH;
  if (r0 >= R) return;
  const int win = it.x & 0xFFFF, L = max(1, it.x >> 16);   // window, cells in the run
  const int nu = TT + L - 1;                      // planes of the run's block
  const WinDev<float> w = wins[win];
  if (io) {
    Out = io[win].Out;
    ldo = io[win].ldo;
    scale = io[win].scale;
  }
  int bnd[kRunCells - 1];                         // first sorted point of cells 1 .. L-1
#pragma unroll
  for (int q = 0; q < kRunCells - 1; ++q)
    bnd[q] = (q + 1 < L) ? __ldg(w.cell_start + it.y + q + 1) : 0x7FFFFFFF;
  const int j0 = it.z, m = it.w;
  int cc[3];
  decode_cell<3>(it.y, w.N, cc);
  auto opnd = [&](int b) { return smem_raw + b * Sh::OPND; };
  float* pb = reinterpret_cast<float*>(smem_raw);   // epilogue partials (operands are free then)
  float* ws = reinterpret_cast<float*>(smem_raw + (2 * Sh::OPND > Sh::PB_BYTES ? 2 * Sh::OPND
                                                                              : Sh::PB_BYTES));
  int* sperm = reinterpret_cast<int*>(ws + kItMP * WPP);
  int* sdelta = sperm + kItMP;                      // cell of each point within the run

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

  // element slot of this thread in every core matrix it writes: row r8 and
  // column k4 of the core, column quad kq (KC / 4 quads), group g of the rows
  const int kq = (tid >> 5) & (KC / 4 - 1), r8 = lane >> 2, k4 = lane & 3, g = tid >> 7;
  const int kk4 = kq * 4 + k4;                   // grid row within the chunk
  const int o = kq * 32 + lane;                  // element offset in the row group 0 core
  const uint32_t idesc = umma_idesc_tf32(kItMP, nu * RH);
  // base pointer of this thread's B elements at grid row kk = (t1, t2):
  // grid + 32 cell(t1, t2, 0) + r0 + r8; row group rg adds 32 (rg / 2) + 8 (rg % 2)
  auto bptr = [&](int kk) -> const float* {
    const int t1 = kk / TT, t2 = kk - (kk / TT) * TT;
    const int64_t cell = ((int64_t)(cc[0] + t1) * w.W + (cc[1] + t2)) * w.W + cc[2];
    return w.grid + cell * rc + r0 + r8;
  };
  auto load_b = [&](int kk, float* gb) {
    const bool krow = kk < Sh::ROWS;
    const float* gp = krow ? bptr(kk) : w.grid;
    if (g == 0) it_load_b<S, 0>(gp, krow, 2 * nu, rc, gb);
    else it_load_b<S, 1>(gp, krow, 2 * nu, rc, gb);
  };
  bool ok = true;
  int gc = 0;                                    // chunks issued so far (all tiles)
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  for (int p0 = 0; p0 < m; p0 += kItMP) {
    const int np = min(kItMP, m - p0);
    // stage the tile's window values and perm indices
    const float* wsrc = w.wts + (int64_t)(j0 + p0) * WPP;
    for (int e = tid; e < np * (WPP / 4); e += kItThreads) cp_async16(ws + e * 4, wsrc + e * 4, 16);
    cp_async_commit();
    for (int e = tid; e < np; e += kItThreads) {
      const int jj = j0 + p0 + e;
      sperm[e] = __ldg(w.perm + jj);
      int delta = 0;
#pragma unroll
      for (int q = 0; q < kRunCells - 1; ++q) delta += jj >= bnd[q];
      sdelta[e] = delta;
    }
    float gb[Sh::BPER];                          // B values of the next chunk
    load_b(kk4, gb);
    cp_async_wait<0>();
    __syncthreads();
    for (int c = 0; c < Sh::NCH; ++c) {
      const int b = gc & 1;
      if (gc >= 2 && !mbar_wait(&bar[b], ((gc - 2) >> 1) & 1, spin)) ok = false;
      float* ahi = reinterpret_cast<float*>(opnd(b));
      float* alo = reinterpret_cast<float*>(opnd(b) + Sh::A_BYTES);
      float* bhi = reinterpret_cast<float*>(opnd(b) + 2 * Sh::A_BYTES);
      float* blo = reinterpret_cast<float*>(opnd(b) + 2 * Sh::A_BYTES + Sh::B_BYTES);
      const int kk = c * KC + kk4;               // this thread's grid row (t1, t2)
      if (g == 0) it_store_b<S, 0>(gb, bhi + o, blo + o);
      else it_store_b<S, 1>(gb, bhi + o, blo + o);
      if (c + 1 < Sh::NCH) load_b(kk + KC, gb);  // next chunk's grid values, in flight
      {
        const bool krow = kk < Sh::ROWS;
        const int t1 = krow ? kk / TT : 0, t2 = krow ? kk - (kk / TT) * TT : 0;
        const float* w1 = ws + r8 * WPP + t1;
        const float* w2 = ws + r8 * WPP + TTP + t2;
        if (g == 0) it_form_a<S, 0>(w1, w2, np, r8, krow, ahi + o, alo + o);
        else it_form_a<S, 1>(w1, w2, np, r8, krow, ahi + o, alo + o);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;");
      ok = __syncthreads_and(ok);                // CTA-wide outcome of the waits so far
      if (!ok) break;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t a0 = umma_desc(smem_u32(ahi), kItLBO, kItSBO);
        const uint64_t a1 = umma_desc(smem_u32(alo), kItLBO, kItSBO);
        const uint64_t b0 = umma_desc(smem_u32(bhi), kItLBO, kItSBO);
        const uint64_t b1 = umma_desc(smem_u32(blo), kItLBO, kItSBO);
#pragma unroll
        for (int s2 = 0; s2 < KC / 8; ++s2) {
          const uint64_t off = (uint64_t)(s2 * 2 * kItLBO) >> 4;
          mma_tf32(tmem, a0 + off, b0 + off, idesc, (c > 0 || s2 > 0) ? 1u : 0u);
          mma_tf32(tmem, a0 + off, b1 + off, idesc, 1u);
          mma_tf32(tmem, a1 + off, b0 + off, idesc, 1u);
        }
        mma_commit(&bar[b]);
      }
      ++gc;
    }
    if (!ok) break;
    // the last commit covers every MMA of the tile (no other phase of its
    // barrier is pending: the wait for the chunk two before it succeeded)
    ok = __syncthreads_and(mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1, spin));
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    {
      // warp w: points 32 (w % 4) .. + 31 (TMEM lanes), t3 half w / 4; partial
      // sums over its t3 range go to shared memory, then four threads per
      // point add the halves and issue one 16-byte atomic each
      const int quarter = warp % 4, part = warp / 4;
      const int p = quarter * 32 + lane;
      float acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
      const int ta = part * nu / 2, tb = (part + 1) * nu / 2;
      const int dp = p < np ? sdelta[p] : 0;
#pragma unroll 1
      for (int t3 = ta; t3 < tb; ++t3) {            // plane of the run's block
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t3 * RH);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];\n"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        const int tp = t3 - dp;                     // this point's tap
        const float ps = (p < np && tp >= 0 && tp < TT) ? ws[p * WPP + 2 * TTP + 2 * tp] : 0.0f;
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = fmaf(ps, __uint_as_float(v[q]), acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) pb[(part * kItMP + p) * 17 + q] = acc[q];
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    {
      const bool vec = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(Out) & 15) == 0);
      for (int e = tid; e < np * 4; e += kItThreads) {
        const int p = e >> 2, c4 = (e & 3) * 4;
        if (r0 + c4 >= R) continue;
        const float* s0 = pb + p * 17 + c4;
        const float* s1 = pb + (kItMP + p) * 17 + c4;
        float4 val = make_float4(scale * (s0[0] + s1[0]), scale * (s0[1] + s1[1]),
                                 scale * (s0[2] + s1[2]), scale * (s0[3] + s1[3]));
        float* dst = Out + (int64_t)sperm[p] * ldo + r0 + c4;
        if (vec && r0 + c4 + 4 <= R) {
          atomicAdd(reinterpret_cast<float4*>(dst), val);
        } else {
          const float vv[4] = {val.x, val.y, val.z, val.w};
          for (int q = 0; q < 4 && r0 + c4 + q < R; ++q) atomicAdd(dst + q, vv[q]);
        }
      }
    }
    __syncthreads();                             // partials, ws and sperm free for the next tile
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok) {
    // a wait expired (the CTA agreed on it): drain the committed MMAs with
    // the fixed bound before TMEM is released, record the timeout
    if (gc > 0) mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1);
    if (tid == 0) atomicOr(err, 2);
  }
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "n"(Sh::TMEM_COLS));
}

template <int S>
cudaError_t interp_tc_s(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                        int64_t n_items, float* Out, int64_t ldo, int R, float scale, int rc,
                        int* err, long long spin, cudaStream_t st) {
  using Sh = TcInterpShape<S>;
  cudaError_t e = cudaFuncSetAttribute(k_interp_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Sh::SMEM);
  if (e != cudaSuccess) return e;
  if (n_items <= 0) return cudaSuccess;
  k_interp_tc<S><<<(unsigned)(rc / 16 * n_items), kItThreads, Sh::SMEM, st>>>(wins, io, items, Out, ldo,
                                                                        R, scale, rc, err, spin);
  return cudaGetLastError();
}

}  // namespace

bool interp_tc_supported(int d, int s, int RC) {
  return d == 3 && (RC == 32 || RC == 16) && (s == 4 || s == 5);
}

cudaError_t interp_items_tc(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                            int64_t n_items, int s, float* Out, int64_t ldo, int R, float scale,
                            int rc, int* err, long long spin, cudaStream_t st) {
  switch (s) {
    case 4: return interp_tc_s<4>(wins, io, items, n_items, Out, ldo, R, scale, rc, err, spin, st);
    case 5: return interp_tc_s<5>(wins, io, items, n_items, Out, ldo, R, scale, rc, err, spin, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace agp
