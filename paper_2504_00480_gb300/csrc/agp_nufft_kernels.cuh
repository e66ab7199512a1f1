#pragma once
// Spreading (adjoint NFFT, Appendix A step 3 transposed) and interpolation
// (NFFT, Appendix A step 3) of the additive-kernel fast summation, Sec. 3.1
// eq. (3.3).
//
// Points are sorted by grid cell at plan time and grouped into work items of
// up to kItemPoints points of one cell; all points of an item touch the same
// (2s)^d block of grid points. The Kaiser-Bessel values of every point are
// precomputed at plan time, [n][d][TTP] with TTP = 2s rounded up to 4 (zero
// padded), in sorted order.
//  * Spreading: one CTA per (item, part of its grid rows) accumulates its
//    rows of the item's (2s)^d block in registers (a lane owns one grid row of
//    2s points x 8 right-hand sides) and adds them to the grid once with
//    vector atomics; point data are staged in shared memory with cp.async,
//    double buffered.
//  * Interpolation: one CTA per (item, slice of right-hand sides) stages the
//    block in shared memory once; a lane evaluates one right-hand side for 8
//    points, so every block value read feeds 8 FMAs, contracting the
//    separable window one dimension at a time.
// Shared-memory reads are arranged so that one warp load is one wavefront
// (32-bit words, broadcast or consecutive): on this part a 128-bit warp load
// costs four wavefronts even when the lanes read the same address.
// Every window and right-hand side of one dimension d runs in one launch.
// This header holds the kernels; agp_nufft_rc<RC>.cu instantiate them for one
// right-hand-side block width RC each (compiled in parallel), agp_nufft.cu
// dispatches.
#include "agp_internal.cuh"

// Compile-time tuning knobs (defaults are the measured best on GB300).
#ifndef AGP_SPREAD_SUB
#define AGP_SPREAD_SUB 64           // points per shared-memory stage of k_spread
#endif
#ifndef AGP_INTERP_T2_UNROLL
#define AGP_INTERP_T2_UNROLL 5      // rows of the block contracted together in k_interp2
#endif
#ifndef AGP_SPREAD_STAGES
#define AGP_SPREAD_STAGES 3         // shared-memory stages in flight in k_spread (2 or 3)
#endif
#ifndef AGP_SPREAD_POINT_UNROLL
#define AGP_SPREAD_POINT_UNROLL 1   // points of a stage processed together in k_spread
#endif
#ifndef AGP_INTERP_RS
#define AGP_INTERP_RS 16            // right-hand sides per CTA of k_interp2 (8 or 16)
#endif
#ifndef AGP_INTERP_ASYNC_W
#define AGP_INTERP_ASYNC_W 1        // stage k_interp2's window values with cp.async
#endif
#ifndef AGP_INTERP_WPS_PAD
#define AGP_INTERP_WPS_PAD 1        // padding of a point's values in k_interp2's shared memory
#endif

namespace agp {
namespace {

template <typename T, int RG>
__device__ __forceinline__ void atomic_add_n(T* p, const T* a) {
  if constexpr (sizeof(T) == 4 && RG % 4 == 0) {
#pragma unroll
    for (int i = 0; i < RG; i += 4)
      atomicAdd(reinterpret_cast<float4*>(p + i), make_float4(a[i], a[i + 1], a[i + 2], a[i + 3]));
  } else {
#pragma unroll
    for (int i = 0; i < RG; ++i) atomicAdd(p + i, a[i]);
  }
}

template <typename T, int K>
__device__ __forceinline__ void load_n(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4 && K % 4 == 0) {
#pragma unroll
    for (int i = 0; i < K; i += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(src + i));
      dst[i] = v.x;
      dst[i + 1] = v.y;
      dst[i + 2] = v.z;
      dst[i + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 8 && K % 2 == 0) {
#pragma unroll
    for (int i = 0; i < K; i += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(src + i));
      dst[i] = v.x;
      dst[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) dst[i] = __ldg(src + i);
  }
}

template <int D>
__device__ __forceinline__ void decode_cell(int cell, int N, int* c) {
  if constexpr (D == 3) {
    c[2] = cell % N;
    c[1] = (cell / N) % N;
    c[0] = cell / (N * N);
  } else if constexpr (D == 2) {
    c[1] = cell % N;
    c[0] = cell / N;
  } else {
    c[0] = cell;
  }
}

constexpr int ttp_of(int s) { return (2 * s + 3) / 4 * 4; }
// values per point: d-1 dimensions of ttp_of(s), then the last dimension's 2s
// taps written twice (pairs (v, v))
constexpr int wpp_of(int d, int s) { return (d - 1) * ttp_of(s) + 4 * s; }

// ---------------------------------------------------------------------------
// cp.async helpers (16-byte global -> shared copies, zero fill beyond src_bytes)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ---------------------------------------------------------------------------
// Packed FP32 pairs: one instruction performs two independent FP32 operations
// (fma.rn.f32x2 / mul.rn.f32x2, each lane of the pair rounded exactly like the
// scalar fmaf / fmulf). Used to halve the issue slots taken by the FMAs of
// spreading and interpolation. The low half of a pair is the first element.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float x2_lo(f32x2 v) { return __uint_as_float((unsigned)(v & 0xFFFFFFFFull)); }
__device__ __forceinline__ float x2_hi(f32x2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// ---------------------------------------------------------------------------
// Spreading: grid[a][r] += sum_j V[perm[j]][r] prod_t psi_t(j, a_t - c_t)
// ---------------------------------------------------------------------------
// One CTA per (work item, part). The item's ROWS grid rows (a row = the 2s
// grid points along the last dimension) are split into PARTS parts (two for
// d = 3 with 32 right-hand sides), so that several CTAs share an SM and one
// CTA's prologue or atomic flush overlaps the FMAs of another. Lane = (one grid row, RG right-hand
// sides), holding 2s x RG accumulators for the whole item. Point data (window
// values and the V rows gathered through perm) are staged SUB points at a
// time in shared memory with cp.async, double buffered; the perm indices of a
// stage are loaded one stage ahead, so their latency hides behind the FMAs.
// Per point a lane reads its row weight (two values for d = 3), the 2s
// last-dimension weights (warp-uniform) and RG values of V, and does 2s x RG
// FMAs (FP32: packed pairs over neighbouring last-dimension taps).
template <typename T, int D, int S, int RC>
struct SpreadShape {
  static constexpr int TT = 2 * S;
  static constexpr int TTP = ttp_of(S);
  static constexpr int RG = (sizeof(T) == 4) ? ((RC % 8 == 0) ? 8 : ((RC % 4 == 0) ? 4 : 1))
                                             : ((RC % 4 == 0) ? 4 : ((RC % 2 == 0) ? 2 : 1));
  static constexpr int NG = RC / RG;
  static constexpr int ROWS = (D == 1) ? 1 : ((D == 2) ? TT : TT * TT);
  static constexpr int PARTS = (D == 3 && ROWS * NG >= 400) ? 2 : 1;
  static constexpr int RPC = ROWS / PARTS;                     // rows per CTA
  static constexpr int LANES = RPC * NG;
  static constexpr int THREADS = (LANES + 31) / 32 * 32;
  static constexpr int SUB = AGP_SPREAD_SUB;                   // points per stage
  static constexpr int WPP = wpp_of(D, S);                     // window values per point
  static constexpr int VROW = (RC * sizeof(T) + 15) / 16 * 16 / sizeof(T);   // padded row
  static constexpr int VCH = (int)(VROW * sizeof(T) / 16);     // 16-byte chunks per V row
  static constexpr int PFN = (SUB * VCH + THREADS - 1) / THREADS;   // chunks per thread
  static constexpr int STAGE = SUB * (WPP + VROW);             // elements per stage
  static constexpr int NST = AGP_SPREAD_STAGES;                // stages in flight
  static constexpr size_t SMEM = NST * STAGE * sizeof(T);
  // CTAs per SM the register budget is sized for (accumulators + ~56 others)
  static constexpr int EST_REGS = (int)(TT * RG * sizeof(T) / 4) + 56;
  static constexpr int MINB_RAW = 65536 / (THREADS * EST_REGS);
  static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 4 ? 4 : MINB_RAW);
};

template <typename T, int D, int S, int RC>
__global__ void __launch_bounds__(SpreadShape<T, D, S, RC>::THREADS, SpreadShape<T, D, S, RC>::MINB)
k_spread(const WinDev<T>* __restrict__ wins, const WinIO<T>* __restrict__ io,
         const int4* __restrict__ items, const T* __restrict__ V, int64_t ldv, int R) {
  using Sh = SpreadShape<T, D, S, RC>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, RG = Sh::RG, NG = Sh::NG;
  constexpr int SUB = Sh::SUB, WPP = Sh::WPP, VROW = Sh::VROW, VCH = Sh::VCH, PFN = Sh::PFN;
  constexpr int E16 = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  const int4 it = items[blockIdx.x / Sh::PARTS];
  const int part = blockIdx.x % Sh::PARTS;
  const WinDev<T> w = wins[it.x];
  if (io) {
    V = io[it.x].V;
    ldv = io[it.x].ldv;
  }
  const bool vec_ok = (ldv % E16 == 0) && ((reinterpret_cast<uintptr_t>(V) & 15) == 0);
  const int j0 = it.z, m = it.w;
  const int tid = threadIdx.x;
  const bool active = tid < Sh::LANES;
  const int g = active ? tid % NG : 0;
  const int row = part * Sh::RPC + (active ? tid / NG : 0);
  // this lane's row: taps (t1, t2) of the first two dimensions (d = 3), t1 (d = 2)
  const int t1 = (D == 3) ? row / TT : row;
  const int t2 = (D == 3) ? row % TT : 0;
  const int col = g * RG;

  // perm indices of the V chunks this thread copies in a stage
  int64_t pf[PFN];
  auto load_perm = [&](int c) {
    const int q0 = c * SUB;
    const int ns = min(SUB, m - q0);
#pragma unroll
    for (int u = 0; u < PFN; ++u) {
      const int e = tid + u * Sh::THREADS;
      pf[u] = (e < ns * VCH) ? (int64_t)__ldg(w.perm + j0 + q0 + e / VCH) : 0;
    }
  };
  // stage loader: window values (contiguous) and V rows (gathered)
  auto stage = [&](int c, int buf) {
    T* ws = sm + buf * Sh::STAGE;
    T* vs = ws + SUB * WPP;
    const int q0 = c * SUB;
    const int ns = min(SUB, m - q0);
    constexpr int WCH = sizeof(T) * WPP / 16;              // 16-byte chunks per point
    const T* wsrc = w.wts + (int64_t)(j0 + q0) * WPP;
    for (int e = tid; e < ns * WCH; e += Sh::THREADS) cp_async16(ws + e * E16, wsrc + e * E16, 16);
    if (vec_ok) {
#pragma unroll
      for (int u = 0; u < PFN; ++u) {
        const int e = tid + u * Sh::THREADS;
        if (e < ns * VCH) {
          const int q = e / VCH, k = e - q * VCH;
          const int c0 = k * E16;
          const int valid = max(0, min(E16, R - c0));
          cp_async16(vs + q * VROW + c0, V + pf[u] * ldv + (valid > 0 ? c0 : 0),
                     valid * (int)sizeof(T));
        }
      }
    } else {
      for (int e = tid; e < ns * VROW; e += Sh::THREADS) {
        const int q = e / VROW, r = e - q * VROW;
        const int64_t i = __ldg(w.perm + j0 + q0 + q);
        vs[e] = (r < R) ? V[i * ldv + r] : T(0);
      }
    }
    cp_async_commit();
  };

  // FP32 with an even number of right-hand sides per lane: packed pairs of
  // neighbouring right-hand sides; otherwise scalar accumulators.
  constexpr bool X2 = sizeof(T) == 4 && RG % 2 == 0;
  constexpr int A2 = X2 ? 1 : TT, A3 = X2 ? 1 : RG;
  constexpr int B2 = X2 ? TT : 1, B3 = X2 ? (RG + 1) / 2 : 1;
  T acc[A2][A3];
  f32x2 acc2[B2][B3];
#pragma unroll
  for (int t = 0; t < A2; ++t)
#pragma unroll
    for (int q = 0; q < A3; ++q) acc[t][q] = T(0);
#pragma unroll
  for (int t = 0; t < B2; ++t)
#pragma unroll
    for (int q = 0; q < B3; ++q) acc2[t][q] = 0ull;

  const int nchunk = (m + SUB - 1) / SUB;
  constexpr int NST = Sh::NST;
  static_assert(NST == 2 || NST == 3, "two or three stages");
  if constexpr (NST == 2) {
    if (vec_ok) load_perm(0);
    stage(0, 0);
    if (vec_ok && nchunk > 1) load_perm(1);
  } else {
    // prologue: chunks 0 and 1 in flight, perm of chunk 2 in registers
    if (vec_ok) load_perm(0);
    stage(0, 0);
    if (nchunk > 1) {
      if (vec_ok) load_perm(1);
      stage(1, 1);
    }
    if (vec_ok && nchunk > 2) load_perm(2);
  }
  for (int c = 0; c < nchunk; ++c) {
    if constexpr (NST == 2) {
      if (c + 1 < nchunk) {
        stage(c + 1, (c + 1) & 1);
        if (vec_ok && c + 2 < nchunk) load_perm(c + 2);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
    } else {
      // chunk c landed (chunk c+1 may still be in flight); after the barrier
      // every thread is done with chunk c-1, whose buffer takes chunk c+2
      if (c + 1 < nchunk) cp_async_wait<1>();
      else cp_async_wait<0>();
      __syncthreads();
      if (c + 2 < nchunk) {
        stage(c + 2, (c + 2) % 3);
        if (vec_ok && c + 3 < nchunk) load_perm(c + 3);
      }
    }
    const T* ws = sm + (c % NST) * Sh::STAGE;
    const T* vs = ws + SUB * WPP;
    const int ns = min(SUB, m - c * SUB);
    constexpr int kPointUnroll = AGP_SPREAD_POINT_UNROLL;
#pragma unroll kPointUnroll
    for (int q = 0; q < ns; ++q) {
      const T* pw = ws + q * WPP;
      T wr;
      if constexpr (D == 3) wr = pw[t1] * pw[TTP + t2];
      else if constexpr (D == 2) wr = pw[t1];
      else wr = T(1);
      T v[RG];
#pragma unroll
      for (int k = 0; k < RG; ++k) v[k] = vs[q * VROW + col + k];
      const T* wl = pw + (D - 1) * TTP;
      if constexpr (X2) {
        // acc2[t][k/2] += (wr v_k, wr v_{k+1}) * (psi_t, psi_t)
        const f32x2 wrr = x2_pack(wr, wr);
        f32x2 a[RG / 2];
#pragma unroll
        for (int kp = 0; kp < RG / 2; ++kp) a[kp] = x2_mul(wrr, x2_pack(v[2 * kp], v[2 * kp + 1]));
#pragma unroll
        for (int t = 0; t < TT; ++t) {
          const f32x2 ww = *reinterpret_cast<const f32x2*>(wl + 2 * t);   // (psi_t, psi_t)
#pragma unroll
          for (int kp = 0; kp < RG / 2; ++kp) acc2[t][kp] = x2_fma(a[kp], ww, acc2[t][kp]);
        }
      } else {
        T a[RG];
#pragma unroll
        for (int k = 0; k < RG; ++k) a[k] = v[k] * wr;
#pragma unroll
        for (int t = 0; t < TT; ++t) {
          const T wv = wl[2 * t];
#pragma unroll
          for (int k = 0; k < RG; ++k) acc[t][k] = fma(a[k], wv, acc[t][k]);
        }
      }
    }
    if constexpr (NST == 2) __syncthreads();   // the buffer of chunk c is refilled at c + 1
  }
  if (!active || col >= R) return;   // padding lanes / padding columns
  int cc[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, cc);
  int64_t base;
  if constexpr (D == 3) base = ((int64_t)(cc[0] + t1) * w.W + (cc[1] + t2)) * w.W + cc[2];
  else if constexpr (D == 2) base = (int64_t)(cc[0] + t1) * w.W + cc[1];
  else base = cc[0];
  T* gp = w.grid + base * RC + col;
  if constexpr (X2) {
#pragma unroll
    for (int t = 0; t < TT; ++t) {
      T a[RG];
#pragma unroll
      for (int kp = 0; kp < RG / 2; ++kp) {
        a[2 * kp] = x2_lo(acc2[t][kp]);
        a[2 * kp + 1] = x2_hi(acc2[t][kp]);
      }
      atomic_add_n<T, RG>(gp + (int64_t)t * RC, a);
    }
  } else {
#pragma unroll
    for (int t = 0; t < TT; ++t) atomic_add_n<T, RG>(gp + (int64_t)t * RC, acc[t]);
  }
}

// FP32 body of the interpolation for one lane (one right-hand side, PP
// points): the PP accumulators are packed in pairs of neighbouring points, so
// each block value h read from shared memory feeds PP/2 paired FMAs with
// (h, h); the lower-dimension weights of two points are paired the same way.
template <int D, int S, int PP, int RS, int WPS, int TTP>
__device__ __forceinline__ void interp_points_x2(const float* __restrict__ ws, int grp, int np,
                                                 const float* __restrict__ hb, float* acc) {
  constexpr int TT = 2 * S, PH = PP / 2;
  f32x2 wl[PH][TT];
#pragma unroll
  for (int j = 0; j < PH; ++j) {
    const int q0 = grp * PP + 2 * j, q1 = q0 + 1;
#pragma unroll
    for (int t = 0; t < TT; ++t)
      wl[j][t] = x2_pack((q0 < np) ? ws[q0 * WPS + (D - 1) * TTP + 2 * t] : 0.0f,
                         (q1 < np) ? ws[q1 * WPS + (D - 1) * TTP + 2 * t] : 0.0f);
  }
  f32x2 a2[PH];
#pragma unroll
  for (int j = 0; j < PH; ++j) a2[j] = 0ull;
  // weight pair of dimension `dim`, tap t, for the points 2j, 2j+1 of the lane
  auto wpair = [&](int j, int dim, int t) {
    const int q0 = grp * PP + 2 * j;
    return x2_pack(ws[q0 * WPS + dim * TTP + t], ws[(q0 + 1) * WPS + dim * TTP + t]);
  };
  if constexpr (D == 1) {
#pragma unroll
    for (int t3 = 0; t3 < TT; ++t3) {
      const float h = hb[t3 * RS];
      const f32x2 hh = x2_pack(h, h);
#pragma unroll
      for (int j = 0; j < PH; ++j) a2[j] = x2_fma(wl[j][t3], hh, a2[j]);
    }
  } else {
    constexpr int N1 = (D == 3) ? TT : 1;
    for (int t1 = 0; t1 < N1; ++t1) {
      f32x2 u1[PH];
#pragma unroll
      for (int j = 0; j < PH; ++j) u1[j] = 0ull;
      for (int t2 = 0; t2 < TT; ++t2) {
        f32x2 u2[PH];
#pragma unroll
        for (int j = 0; j < PH; ++j) u2[j] = 0ull;
        const float* hrow = hb + ((t1 * TT + t2) * TT) * RS;
#pragma unroll
        for (int t3 = 0; t3 < TT; ++t3) {
          const float h = hrow[t3 * RS];
          const f32x2 hh = x2_pack(h, h);
#pragma unroll
          for (int j = 0; j < PH; ++j) u2[j] = x2_fma(wl[j][t3], hh, u2[j]);
        }
#pragma unroll
        for (int j = 0; j < PH; ++j) u1[j] = x2_fma(wpair(j, D - 2, t2), u2[j], u1[j]);
      }
      if constexpr (D == 3) {
#pragma unroll
        for (int j = 0; j < PH; ++j) a2[j] = x2_fma(wpair(j, 0, t1), u1[j], a2[j]);
      } else {
#pragma unroll
        for (int j = 0; j < PH; ++j) a2[j] = u1[j];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PH; ++j) {
    acc[2 * j] = x2_lo(a2[j]);
    acc[2 * j + 1] = x2_hi(a2[j]);
  }
}

template <typename T, int D, int S, int RC>
struct InterpShape {
  static constexpr int TT = 2 * S;
  static constexpr int TTP = ttp_of(S);
  static constexpr int RS = (RC >= 16) ? 16 : RC;               // right-hand sides per CTA
  static constexpr int GROUPS_PER_WARP = 32 / RS;               // point groups per warp
  static constexpr int THREADS = 128;
  static constexpr int PP = (sizeof(T) == 4) ? 8 : 4;           // points per lane
  static constexpr int NGRP = THREADS / RS;                     // point groups per CTA
  static constexpr int PTS = NGRP * PP;                         // points per pass
  static constexpr int BLK = (D == 1) ? TT : ((D == 2) ? TT * TT : TT * TT * TT);
  static constexpr int WPP = wpp_of(D, S);
  // shared-memory stride of a point's window values: odd, so that the point
  // groups of one warp (PP points apart) read different banks
  static constexpr int WPS = WPP + 1;
  static constexpr int CPC = (int)(RS * sizeof(T) / 16);       // 16-byte chunks per staged cell
  static constexpr size_t SMEM = sizeof(T) * ((size_t)BLK * RS + (size_t)PTS * WPS);
};

template <typename T, int D, int S, int RC>
__global__ void __launch_bounds__(128)
k_interp(const WinDev<T>* __restrict__ wins, const WinIO<T>* __restrict__ io,
         const int4* __restrict__ items, T* __restrict__ Out, int64_t ldo, int R, T scale) {
  using Sh = InterpShape<T, D, S, RC>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, RS = Sh::RS, PP = Sh::PP, PTS = Sh::PTS;
  constexpr int BLK = Sh::BLK, WPP = Sh::WPP, WPS = Sh::WPS, CPC = Sh::CPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Hs = reinterpret_cast<T*>(smem_raw);   // [BLK][RS]
  T* ws = Hs + BLK * RS;                     // [PTS][WPS]

  const int rs0 = blockIdx.y * RS;
  if (rs0 >= R) return;
  const int4 it = items[blockIdx.x];
  const WinDev<T> w = wins[it.x];
  if (io) {
    Out = io[it.x].Out;
    ldo = io[it.x].ldo;
    scale = io[it.x].scale;
  }
  const int j0 = it.z, m = it.w;
  int c[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, c);
  const int tid = threadIdx.x;

  // Stage the item's (2s)^d block, columns rs0 .. rs0+RS-1 (asynchronous
  // 16-byte copies when a cell's slice is a whole number of 16-byte chunks).
  auto cell_index = [&](int ci) -> int64_t {
    if constexpr (D == 3) {
      const int a3 = ci % TT, a2 = (ci / TT) % TT, a1 = ci / (TT * TT);
      return ((int64_t)(c[0] + a1) * w.W + (c[1] + a2)) * w.W + (c[2] + a3);
    } else if constexpr (D == 2) {
      const int a2 = ci % TT, a1 = ci / TT;
      return (int64_t)(c[0] + a1) * w.W + (c[1] + a2);
    } else {
      return c[0] + ci;
    }
  };
  if constexpr (CPC >= 1 && RS * sizeof(T) % 16 == 0) {
    constexpr int E16 = 16 / sizeof(T);
    for (int e = tid; e < BLK * CPC; e += Sh::THREADS) {
      const int ci = e / CPC, k = e - ci * CPC;
      cp_async16(Hs + ci * RS + k * E16, w.grid + cell_index(ci) * RC + rs0 + k * E16, 16);
    }
    cp_async_commit();
  } else {
    for (int e = tid; e < BLK * RS; e += Sh::THREADS) {
      const int ci = e / RS, r = e - ci * RS;
      Hs[e] = w.grid[cell_index(ci) * RC + rs0 + r];
    }
  }

  const int r = tid % RS;                   // right-hand side of this lane
  const int grp = tid / RS;                 // point group: points grp*PP .. grp*PP+PP-1
  const int warp_first_grp = (tid / 32) * Sh::GROUPS_PER_WARP;
  for (int p0 = 0; p0 < m; p0 += PTS) {
    const int np = min(PTS, m - p0);
    __syncthreads();                          // previous pass done with ws
    for (int e = tid; e < np * WPP; e += Sh::THREADS) {
      const int q = e / WPP;
      ws[q * WPS + (e - q * WPP)] = __ldg(w.wts + (int64_t)(j0 + p0) * WPP + e);
    }
    cp_async_wait<0>();                       // the staged block has landed (first pass)
    __syncthreads();
    if (warp_first_grp * PP >= np) continue;  // no point of this pass in this warp

    T acc[PP];
#pragma unroll
    for (int k = 0; k < PP; ++k) acc[k] = T(0);
    const T* hb = Hs + r;
    if constexpr (sizeof(T) == 4) {
      interp_points_x2<D, S, PP, RS, WPS, TTP>(ws, grp, np, hb, acc);
    } else {
    T wl[PP][TT];
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int q = grp * PP + k;
#pragma unroll
      for (int t = 0; t < TT; ++t) wl[k][t] = (q < np) ? ws[q * WPS + (D - 1) * TTP + 2 * t] : T(0);
    }
    if constexpr (D == 1) {
#pragma unroll
      for (int t3 = 0; t3 < TT; ++t3) {
        const T h = hb[t3 * RS];
#pragma unroll
        for (int k = 0; k < PP; ++k) acc[k] = fma(wl[k][t3], h, acc[k]);
      }
    } else {
      constexpr int N1 = (D == 3) ? TT : 1;
      for (int t1 = 0; t1 < N1; ++t1) {
        T u1[PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) u1[k] = T(0);
        for (int t2 = 0; t2 < TT; ++t2) {
          T u2[PP];
#pragma unroll
          for (int k = 0; k < PP; ++k) u2[k] = T(0);
          const T* hrow = hb + ((t1 * TT + t2) * TT) * RS;
#pragma unroll
          for (int t3 = 0; t3 < TT; ++t3) {
            const T h = hrow[t3 * RS];
#pragma unroll
            for (int k = 0; k < PP; ++k) u2[k] = fma(wl[k][t3], h, u2[k]);
          }
#pragma unroll
          for (int k = 0; k < PP; ++k) {
            const int q = min(grp * PP + k, PTS - 1);
            u1[k] = fma(ws[q * WPS + (D - 2) * TTP + t2], u2[k], u1[k]);
          }
        }
        if constexpr (D == 3) {
#pragma unroll
          for (int k = 0; k < PP; ++k) {
            const int q = min(grp * PP + k, PTS - 1);
            acc[k] = fma(ws[q * WPS + t1], u1[k], acc[k]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < PP; ++k) acc[k] = u1[k];
        }
      }
    }
    }
    if (rs0 + r < R) {
#pragma unroll
      for (int k = 0; k < PP; ++k) {
        const int q = grp * PP + k;
        if (q < np) {
          const int64_t i = __ldg(w.perm + j0 + p0 + q);
          atomicAdd(Out + i * ldo + rs0 + r, scale * acc[k]);
        }
      }
    }
  }
}

// Interpolation of one right-hand side, one thread per point. A CTA takes
// kPtsItems consecutive work items and numbers their points through a prefix
// sum in shared memory; each point reads its (2s)^d grid block straight from
// the grid (a cell's block is shared by the cell's points through the L1
// cache) and contracts it one dimension at a time. For sparse cells (a few
// points per work item) this replaces a CTA per item that stages a whole
// block for two or three points.
constexpr int kPtsItems = 64;

template <typename T, int D, int S>
__global__ void __launch_bounds__(128)
k_interp_pts(const WinDev<T>* __restrict__ wins, const WinIO<T>* __restrict__ io,
             const int4* __restrict__ items, int64_t n_items, T* __restrict__ Out, int64_t ldo,
             T scale) {
  constexpr int TT = 2 * S, TTP = ttp_of(S), WPP = wpp_of(D, S);
  __shared__ int4 its[kPtsItems];
  __shared__ int pre[kPtsItems + 1];
  const int64_t i0 = (int64_t)blockIdx.x * kPtsItems;
  const int ni = (int)(n_items - i0 < kPtsItems ? n_items - i0 : kPtsItems);
  if (threadIdx.x < ni) its[threadIdx.x] = items[i0 + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < ni; ++q) {
      pre[q] = acc;
      acc += its[q].w;
    }
    pre[ni] = acc;
  }
  __syncthreads();
  const int P = pre[ni];
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    int lo = 0, hi = ni - 1;                   // the item holding point p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    const int4 it = its[lo];
    const WinDev<T>& w = wins[it.x];
    const int j = it.z + (p - pre[lo]);
    int c[3] = {0, 0, 0};
    decode_cell<D>(it.y, w.N, c);
    const T* pw = w.wts + (int64_t)j * WPP;
    const T* pl = pw + (D - 1) * TTP;          // last dimension: (v, v) pairs
    const int64_t W = w.W;
    T acc = T(0);
    if constexpr (D == 3) {
      for (int t1 = 0; t1 < TT; ++t1) {
        T u1 = T(0);
        for (int t2 = 0; t2 < TT; ++t2) {
          const T* g = w.grid + ((c[0] + t1) * W + (c[1] + t2)) * W + c[2];
          T u2 = T(0);
#pragma unroll
          for (int t3 = 0; t3 < TT; ++t3) u2 = fma(pl[2 * t3], g[t3], u2);
          u1 = fma(pw[TTP + t2], u2, u1);
        }
        acc = fma(pw[t1], u1, acc);
      }
    } else if constexpr (D == 2) {
      for (int t1 = 0; t1 < TT; ++t1) {
        const T* g = w.grid + (c[0] + t1) * W + c[1];
        T u = T(0);
#pragma unroll
        for (int t2 = 0; t2 < TT; ++t2) u = fma(pl[2 * t2], g[t2], u);
        acc = fma(pw[t1], u, acc);
      }
    } else {
#pragma unroll
      for (int t = 0; t < TT; ++t) acc = fma(pl[2 * t], w.grid[c[0] + t], acc);
    }
    T* out = Out;
    int64_t ld = ldo;
    T sc = scale;
    if (io) {
      out = io[it.x].Out;
      ld = io[it.x].ldo;
      sc = io[it.x].scale;
    }
    atomicAdd(out + (int64_t)__ldg(w.perm + j) * ld, sc * acc);
  }
}

// FP32 interpolation with pairs of right-hand sides: one CTA per (work item,
// slice of RS right-hand sides), block staged as in k_interp. Lane = (a pair
// of neighbouring right-hand sides, PP = 4 points): a block pair read with one
// 64-bit shared load feeds PP packed FMAs directly, against the points'
// last-dimension weights held in registers as (psi, psi) pairs.
template <int D, int S, int RC>
struct Interp2Shape {
  static constexpr int TT = 2 * S;
  static constexpr int TTP = ttp_of(S);
  static constexpr int RS = (RC % 16 == 0) ? AGP_INTERP_RS : 8;  // right-hand sides per CTA
  static constexpr int RP = RS / 2;                             // pairs per point group
  static constexpr int THREADS = 128;
  static constexpr int PP = 4;                                  // points per lane
  static constexpr int NGRP = THREADS / RP;                     // point groups per CTA
  static constexpr int GPW = 32 / RP;                           // point groups per warp
  static constexpr int PTS = NGRP * PP;                         // points per pass
  static constexpr int BLK = (D == 1) ? TT : ((D == 2) ? TT * TT : TT * TT * TT);
  static constexpr int WPP = wpp_of(D, S);
  // stride of a point's values in shared memory (WPP is a multiple of 4; an
  // odd stride puts the point groups of a warp, PP points apart, on
  // different banks)
  static constexpr int WPS = WPP + AGP_INTERP_WPS_PAD;
  static constexpr int CPC = RS * 4 / 16;                      // 16-byte chunks per staged cell
  static constexpr size_t SMEM = sizeof(float) * ((size_t)BLK * RS + (size_t)PTS * WPS);
};

template <int D, int S, int RC>
__global__ void __launch_bounds__(128)
k_interp2(const WinDev<float>* __restrict__ wins, const WinIO<float>* __restrict__ io,
          const int4* __restrict__ items, float* __restrict__ Out, int64_t ldo, int R, float scale) {
  using Sh = Interp2Shape<D, S, RC>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, RS = Sh::RS, RP = Sh::RP, PP = Sh::PP, PTS = Sh::PTS;
  constexpr int BLK = Sh::BLK, WPP = Sh::WPP, WPS = Sh::WPS, CPC = Sh::CPC;
  static_assert(RS % 4 == 0, "RS must be a multiple of 4");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Hs = reinterpret_cast<float*>(smem_raw);   // [BLK][RS]
  float* ws = Hs + BLK * RS;                         // [PTS][WPS]

  const int rs0 = blockIdx.y * RS;
  if (rs0 >= R) return;
  const int4 it = items[blockIdx.x];
  const WinDev<float> w = wins[it.x];
  if (io) {
    Out = io[it.x].Out;
    ldo = io[it.x].ldo;
    scale = io[it.x].scale;
  }
  const int j0 = it.z, m = it.w;
  int c[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, c);
  const int tid = threadIdx.x;

  // stage the item's (2s)^d block, columns rs0 .. rs0+RS-1
  for (int e = tid; e < BLK * CPC; e += Sh::THREADS) {
    const int ci = e / CPC, k = e - ci * CPC;
    int64_t cell;
    if constexpr (D == 3) {
      const int a3 = ci % TT, a2 = (ci / TT) % TT, a1 = ci / (TT * TT);
      cell = ((int64_t)(c[0] + a1) * w.W + (c[1] + a2)) * w.W + (c[2] + a3);
    } else if constexpr (D == 2) {
      cell = (int64_t)(c[0] + ci / TT) * w.W + (c[1] + ci % TT);
    } else {
      cell = c[0] + ci;
    }
    cp_async16(Hs + ci * RS + k * 4, w.grid + cell * RC + rs0 + k * 4, 16);
  }
  cp_async_commit();

  const int rp = tid % RP;                  // right-hand sides rs0 + 2 rp, +1
  const int grp = tid / RP;                 // points grp*PP .. grp*PP+PP-1 of a pass
  const int warp_first_grp = (tid / 32) * Sh::GPW;
  const int col = rs0 + 2 * rp;
  const bool vec_out = ((ldo & 1) == 0) && ((reinterpret_cast<uintptr_t>(Out) & 7) == 0);
  for (int p0 = 0; p0 < m; p0 += PTS) {
    const int np = min(PTS, m - p0);
    __syncthreads();                          // previous pass done with ws
    // window values of this pass by asynchronous 4-byte copies: in the first
    // pass they travel together with the block
    for (int e = tid; e < np * WPP; e += Sh::THREADS) {
      const int q = e / WPP;
      if constexpr (AGP_INTERP_ASYNC_W)
        cp_async4(ws + q * WPS + (e - q * WPP), w.wts + (int64_t)(j0 + p0) * WPP + e);
      else
        ws[q * WPS + (e - q * WPP)] = __ldg(w.wts + (int64_t)(j0 + p0) * WPP + e);
    }
    cp_async_commit();
    cp_async_wait<0>();                       // block (first pass) and window values landed
    __syncthreads();
    if (warp_first_grp * PP >= np) continue;  // no point of this pass in this warp

    f32x2 wl[PP][TT];
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int q = grp * PP + k;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const float v = (q < np) ? ws[q * WPS + (D - 1) * TTP + 2 * t] : 0.0f;
        wl[k][t] = x2_pack(v, v);
      }
    }
    auto wdup = [&](int k, int dim, int t) {
      const float v = ws[min(grp * PP + k, PTS - 1) * WPS + dim * TTP + t];
      return x2_pack(v, v);
    };
    f32x2 acc[PP];
#pragma unroll
    for (int k = 0; k < PP; ++k) acc[k] = 0ull;
    const float* hb = Hs + 2 * rp;
    if constexpr (D == 1) {
#pragma unroll
      for (int t3 = 0; t3 < TT; ++t3) {
        const f32x2 h = *reinterpret_cast<const f32x2*>(hb + t3 * RS);
#pragma unroll
        for (int k = 0; k < PP; ++k) acc[k] = x2_fma(wl[k][t3], h, acc[k]);
      }
    } else {
      constexpr int N1 = (D == 3) ? TT : 1;
      for (int t1 = 0; t1 < N1; ++t1) {
        f32x2 u1[PP];
#pragma unroll
        for (int k = 0; k < PP; ++k) u1[k] = 0ull;
        constexpr int kT2Unroll = AGP_INTERP_T2_UNROLL;
#pragma unroll kT2Unroll
        for (int t2 = 0; t2 < TT; ++t2) {
          f32x2 u2[PP];
#pragma unroll
          for (int k = 0; k < PP; ++k) u2[k] = 0ull;
          const float* hrow = hb + ((t1 * TT + t2) * TT) * RS;
#pragma unroll
          for (int t3 = 0; t3 < TT; ++t3) {
            const f32x2 h = *reinterpret_cast<const f32x2*>(hrow + t3 * RS);
#pragma unroll
            for (int k = 0; k < PP; ++k) u2[k] = x2_fma(wl[k][t3], h, u2[k]);
          }
#pragma unroll
          for (int k = 0; k < PP; ++k) u1[k] = x2_fma(wdup(k, D - 2, t2), u2[k], u1[k]);
        }
        if constexpr (D == 3) {
#pragma unroll
          for (int k = 0; k < PP; ++k) acc[k] = x2_fma(wdup(k, 0, t1), u1[k], acc[k]);
        } else {
#pragma unroll
          for (int k = 0; k < PP; ++k) acc[k] = u1[k];
        }
      }
    }
    if (col < R) {
#pragma unroll
      for (int k = 0; k < PP; ++k) {
        const int q = grp * PP + k;
        if (q < np) {
          const int64_t i = __ldg(w.perm + j0 + p0 + q);
          const float lo = scale * x2_lo(acc[k]), hi = scale * x2_hi(acc[k]);
          float* o = Out + i * ldo + col;
          if (vec_out && col + 1 < R) {
            atomicAdd(reinterpret_cast<float2*>(o), make_float2(lo, hi));
          } else {
            atomicAdd(o, lo);
            if (col + 1 < R) atomicAdd(o + 1, hi);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Spreading of one right-hand side by rows of cells (d = 2, 3)
// ---------------------------------------------------------------------------
// A row is the cells that share every coordinate but the last; its points
// touch a (2s)^(d-1) x (N + 2s - 1) block of the grid. A CTA takes
// kRowItems consecutive work items (cells in order, so mostly one row),
// splits them into segments of one (window, row) and accumulates each
// segment's block in shared memory: the segment's points (a contiguous range
// of sorted points) are staged kRowStage at a time -- window values with
// coalesced loads, the right-hand side through the permutation, each point's
// cell -- and a thread that owns one block row (t1, t2) adds each point's 2s
// products into its own row, so the accumulation needs no atomics; GROUPS
// groups of threads take every GROUPS-th point into copies of the block,
// which are summed when the block goes into the grid (global atomics for its
// non-zero values only). For sparse cells this replaces a CTA and (2s)^d
// global atomics per cell with about one atomic per block value and row.
constexpr int kRowItems = 32;
constexpr int kRowMaxN = 64;                  // the largest grid size N of a plan
constexpr int kRowThreads = 256;
constexpr int kRowStage = 128;                // points staged at a time

template <typename T, int D, int S>
struct RowShape {
  static constexpr int TT = 2 * S;
  static constexpr int ROWS = (D == 3) ? TT * TT : TT;           // block rows
  static constexpr int ROWSP = (ROWS + 31) / 32 * 32;            // threads per group
  static constexpr int GROUPS = kRowThreads / ROWSP;
  static constexpr int BWMAX = kRowMaxN + TT - 1;                // block width (cells + taps)
  static constexpr int WPP = wpp_of(D, S);
  static constexpr size_t BLK = (size_t)GROUPS * ROWS * BWMAX;   // elements of the block copies
  static constexpr size_t SMEM = sizeof(T) * (BLK + (size_t)kRowStage * (WPP + 1)) +
                                 sizeof(int) * kRowStage;
  static_assert(GROUPS >= 1, "block rows per group");
};

template <typename T, int D, int S>
__global__ void __launch_bounds__(kRowThreads)
k_spread_rows(const WinDev<T>* __restrict__ wins, const WinIO<T>* __restrict__ io,
              const int4* __restrict__ items, int64_t n_items, const T* __restrict__ V,
              int64_t ldv) {
  using Sh = RowShape<T, D, S>;
  constexpr int TT = Sh::TT, TTP = ttp_of(S), WPP = Sh::WPP, ROWS = Sh::ROWS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* blk = reinterpret_cast<T*>(smem_raw);      // [GROUPS][ROWS][BW]
  T* sw = blk + Sh::BLK;                        // [kRowStage][WPP] staged window values
  T* sv = sw + kRowStage * WPP;                 // [kRowStage] right-hand side values
  int* sc = reinterpret_cast<int*>(sv + kRowStage);   // [kRowStage] cell along the last dim
  __shared__ int4 its[kRowItems];
  __shared__ int pre[kRowItems + 1];
  const int64_t i0 = (int64_t)blockIdx.x * kRowItems;
  const int ni = (int)(n_items - i0 < kRowItems ? n_items - i0 : kRowItems);
  if (threadIdx.x < ni) its[threadIdx.x] = items[i0 + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < ni; ++q) {
      pre[q] = acc;
      acc += its[q].w;
    }
    pre[ni] = acc;
  }
  __syncthreads();
  const int grp = threadIdx.x / Sh::ROWSP, row = threadIdx.x - grp * Sh::ROWSP;
  const bool active = grp < Sh::GROUPS && row < ROWS;
  const int t1 = (D == 3) ? row / TT : row, t2 = (D == 3) ? row - (row / TT) * TT : 0;
  int sa = 0;
  while (sa < ni) {
    // the segment [sa, sb): items of one window and one row of cells, whose
    // points are the contiguous sorted range j0 .. j0 + P - 1
    const int win = its[sa].x;
    const WinDev<T>& w = wins[win];
    const int N = w.N, crow = its[sa].y / N;
    int sb = sa + 1;
    while (sb < ni && its[sb].x == win && its[sb].y / N == crow) ++sb;
    const int BW = N + TT - 1;
    const int j0 = its[sa].z, P = pre[sb] - pre[sa];
    for (int e = threadIdx.x; e < Sh::GROUPS * ROWS * BW; e += blockDim.x) blk[e] = T(0);
    const T* Vw = V;
    int64_t ld = ldv;
    if (io) {
      Vw = io[win].V;
      ld = io[win].ldv;
    }
    T* b = blk + ((int64_t)(active ? grp : 0) * ROWS + row) * BW;
    for (int q0 = 0; q0 < P; q0 += kRowStage) {
      const int ns = min(kRowStage, P - q0);
      __syncthreads();                          // the previous stage is consumed, the block zeroed
      const T* src = w.wts + (int64_t)(j0 + q0) * WPP;
      for (int e = threadIdx.x; e < ns * WPP; e += blockDim.x) sw[e] = src[e];
      for (int q = threadIdx.x; q < ns; q += blockDim.x) {
        const int pp = pre[sa] + q0 + q;
        int lo = sa, hi = sb - 1;               // the item holding point pp
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= pp) lo = mid;
          else hi = mid - 1;
        }
        sc[q] = its[lo].y - crow * N;
        sv[q] = Vw[(int64_t)__ldg(w.perm + j0 + q0 + q) * ld];
      }
      __syncthreads();
      if (active) {
        for (int q = grp; q < ns; q += Sh::GROUPS) {
          const T* pw = sw + q * WPP;
          const T a = (D == 3) ? pw[t1] * pw[TTP + t2] * sv[q] : pw[t1] * sv[q];
          const T* pl = pw + (D - 1) * TTP;     // last dimension: (v, v) pairs
          T* bq = b + sc[q];
#pragma unroll
          for (int t3 = 0; t3 < TT; ++t3) bq[t3] = fma(a, pl[2 * t3], bq[t3]);
        }
      }
    }
    __syncthreads();
    // the block (summed over the groups) into the grid: rows (c0 + t1, c1 + t2)
    const int64_t W = w.W;
    int c0 = 0, c1 = 0;
    if constexpr (D == 3) {
      c0 = crow / N;
      c1 = crow - c0 * N;
    } else {
      c0 = crow;
    }
    for (int e = threadIdx.x; e < ROWS * BW; e += blockDim.x) {
      T x = T(0);
#pragma unroll
      for (int q = 0; q < Sh::GROUPS; ++q) x += blk[(int64_t)q * ROWS * BW + e];
      if (x == T(0)) continue;
      const int r = e / BW, u = e - r * BW;
      int64_t gi;
      if constexpr (D == 3) {
        gi = ((c0 + r / TT) * W + (c1 + r % TT)) * W + u;
      } else {
        gi = (c0 + r) * W + u;
      }
      atomicAdd(w.grid + gi, x);
    }
    __syncthreads();
    sa = sb;
  }
}

// ---------------------------------------------------------------------------
// Dispatch over (d, s, RC)
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int RC>
cudaError_t spread_one(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                       int64_t n_items, const T* V, int64_t ldv, int R, cudaStream_t st) {
  using Sh = SpreadShape<T, D, S, RC>;
  if (n_items <= 0) return cudaSuccess;
  if constexpr (RC == 1 && D >= 2) {
    using Rs = RowShape<T, D, S>;
    static bool rattr_set = false;   // per instantiation
    if (!rattr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_spread_rows<T, D, S>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Rs::SMEM);
      if (e != cudaSuccess) return e;
      rattr_set = true;
    }
    const unsigned grid = (unsigned)((n_items + kRowItems - 1) / kRowItems);
    k_spread_rows<T, D, S><<<grid, kRowThreads, Rs::SMEM, st>>>(wins, io, items, n_items, V, ldv);
    return cudaGetLastError();
  }
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_spread<T, D, S, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_spread<T, D, S, RC><<<(unsigned)(n_items * Sh::PARTS), Sh::THREADS, Sh::SMEM, st>>>(
      wins, io, items, V, ldv, R);
  return cudaGetLastError();
}

template <typename T, int D, int S, int RC>
cudaError_t interp_one(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                       int64_t n_items, T* Out, int64_t ldo, int R, T scale, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4 && RC % 8 == 0) {
    using Sh2 = Interp2Shape<D, S, RC>;
    static bool attr2_set = false;   // per instantiation
    if (!attr2_set) {
      cudaError_t e = cudaFuncSetAttribute(k_interp2<D, S, RC>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Sh2::SMEM);
      if (e != cudaSuccess) return e;
      attr2_set = true;
    }
    dim3 grid((unsigned)n_items, (RC + Sh2::RS - 1) / Sh2::RS);
    k_interp2<D, S, RC><<<grid, Sh2::THREADS, Sh2::SMEM, st>>>(wins, io, items, Out, ldo, R, scale);
    return cudaGetLastError();
  } else if constexpr (RC == 1) {
    const unsigned grid = (unsigned)((n_items + kPtsItems - 1) / kPtsItems);
    k_interp_pts<T, D, S><<<grid, 128, 0, st>>>(wins, io, items, n_items, Out, ldo, scale);
    return cudaGetLastError();
  } else {
    using Sh = InterpShape<T, D, S, RC>;
    static bool attr_set = false;   // per instantiation
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_interp<T, D, S, RC>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Sh::SMEM);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    dim3 grid((unsigned)n_items, (RC + Sh::RS - 1) / Sh::RS);
    k_interp<T, D, S, RC><<<grid, Sh::THREADS, Sh::SMEM, st>>>(wins, io, items, Out, ldo, R, scale);
    return cudaGetLastError();
  }
}

}  // namespace
}  // namespace agp

namespace agp {
// Dispatch over (d, s) for one (precision, block width RC); defined in
// agp_nufft_rc<RC>.cu.
#define AGP_NUFFT_RC_DECL(T, RC)                                                              \
  cudaError_t spread_rc##RC(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,     \
                            int64_t n_items, int d, int s, const T* V, int64_t ldv, int R,    \
                            cudaStream_t st);                                                 \
  cudaError_t interp_rc##RC(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,     \
                            int64_t n_items, int d, int s, T* Out, int64_t ldo, int R,        \
                            T scale, cudaStream_t st);
AGP_NUFFT_RC_DECL(float, 1)
AGP_NUFFT_RC_DECL(float, 8)
AGP_NUFFT_RC_DECL(float, 16)
AGP_NUFFT_RC_DECL(float, 24)
AGP_NUFFT_RC_DECL(float, 32)
AGP_NUFFT_RC_DECL(double, 1)
AGP_NUFFT_RC_DECL(double, 4)

// Definition used by the agp_nufft_rc<RC>.cu files.
#define AGP_NUFFT_RC_DEFINE(T, RC)                                                            \
  cudaError_t spread_rc##RC(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,     \
                            int64_t n_items, int d, int s, const T* V, int64_t ldv, int R,    \
                            cudaStream_t st) {                                                \
    return nufft_dispatch<T, RC>::spread(wins, io, items, n_items, d, s, V, ldv, R, st);      \
  }                                                                                           \
  cudaError_t interp_rc##RC(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,     \
                            int64_t n_items, int d, int s, T* Out, int64_t ldo, int R,        \
                            T scale, cudaStream_t st) {                                       \
    return nufft_dispatch<T, RC>::interp(wins, io, items, n_items, d, s, Out, ldo, R, scale,  \
                                         st);                                                 \
  }

namespace {
template <typename T, int RC>
struct nufft_dispatch {
  template <int D>
  static cudaError_t spread_d(int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                              int64_t n_items, const T* V, int64_t ldv, int R, cudaStream_t st) {
    switch (s) {
      case 2: return spread_one<T, D, 2, RC>(wins, io, items, n_items, V, ldv, R, st);
      case 3: return spread_one<T, D, 3, RC>(wins, io, items, n_items, V, ldv, R, st);
      case 4: return spread_one<T, D, 4, RC>(wins, io, items, n_items, V, ldv, R, st);
      case 5: return spread_one<T, D, 5, RC>(wins, io, items, n_items, V, ldv, R, st);
      case 6: return spread_one<T, D, 6, RC>(wins, io, items, n_items, V, ldv, R, st);
    }
    return cudaErrorInvalidValue;
  }
  template <int D>
  static cudaError_t interp_d(int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                              int64_t n_items, T* Out, int64_t ldo, int R, T scale,
                              cudaStream_t st) {
    switch (s) {
      case 2: return interp_one<T, D, 2, RC>(wins, io, items, n_items, Out, ldo, R, scale, st);
      case 3: return interp_one<T, D, 3, RC>(wins, io, items, n_items, Out, ldo, R, scale, st);
      case 4: return interp_one<T, D, 4, RC>(wins, io, items, n_items, Out, ldo, R, scale, st);
      case 5: return interp_one<T, D, 5, RC>(wins, io, items, n_items, Out, ldo, R, scale, st);
      case 6: return interp_one<T, D, 6, RC>(wins, io, items, n_items, Out, ldo, R, scale, st);
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t spread(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                            int64_t n_items, int d, int s, const T* V, int64_t ldv, int R,
                            cudaStream_t st) {
    if (d == 1) return spread_d<1>(s, wins, io, items, n_items, V, ldv, R, st);
    if (d == 2) return spread_d<2>(s, wins, io, items, n_items, V, ldv, R, st);
    if (d == 3) return spread_d<3>(s, wins, io, items, n_items, V, ldv, R, st);
    return cudaErrorInvalidValue;
  }
  static cudaError_t interp(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                            int64_t n_items, int d, int s, T* Out, int64_t ldo, int R, T scale,
                            cudaStream_t st) {
    if (d == 1) return interp_d<1>(s, wins, io, items, n_items, Out, ldo, R, scale, st);
    if (d == 2) return interp_d<2>(s, wins, io, items, n_items, Out, ldo, R, scale, st);
    if (d == 3) return interp_d<3>(s, wins, io, items, n_items, Out, ldo, R, scale, st);
    return cudaErrorInvalidValue;
  }
};
}  // namespace
}  // namespace agp
