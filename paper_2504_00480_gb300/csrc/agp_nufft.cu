// Spreading (adjoint NFFT, Appendix A step 3 transposed) and interpolation
// (NFFT, Appendix A step 3) of the additive-kernel fast summation, Sec. 3.1
// eq. (3.3).
//
// Points are sorted by grid cell at plan time and grouped into work items of
// up to kItemPoints points of one cell; all points of an item touch the same
// (2s)^d block of grid points. The Kaiser-Bessel values of every point are
// precomputed at plan time, [n][d][TTP] with TTP = 2s rounded up to 4 (zero
// padded), in sorted order.
//  * Spreading: one CTA per item accumulates the item's whole (2s)^d block in
//    registers (a lane owns two grid rows of 2s points x 8 right-hand sides)
//    and adds it to the grid once with vector atomics; point data are staged
//    in shared memory with cp.async, double buffered.
//  * Interpolation: one CTA per (item, slice of right-hand sides) stages the
//    block in shared memory once; a lane evaluates one right-hand side for 8
//    points, so every block value read feeds 8 FMAs, contracting the
//    separable window one dimension at a time.
// Shared-memory reads are arranged so that one warp load is one wavefront
// (32-bit words, broadcast or consecutive): on this part a 128-bit warp load
// costs four wavefronts even when the lanes read the same address.
// Every window and right-hand side of one dimension d runs in one launch.
#include "agp_internal.cuh"

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

// ---------------------------------------------------------------------------
// cp.async helpers (16-byte global -> shared copies, zero fill beyond src_bytes)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ---------------------------------------------------------------------------
// Spreading: grid[a][r] += sum_j V[perm[j]][r] prod_t psi_t(j, a_t - c_t)
// ---------------------------------------------------------------------------
// One CTA per work item. Lane = (RPL grid rows, RG right-hand sides); a row is
// the 2s grid points along the last dimension, so a lane holds RPL x 2s x RG
// accumulators for the whole item. Point data (window values and the V rows
// gathered through perm) are staged SUB points at a time in shared memory
// with cp.async, double buffered. Per point each lane reads its row weights,
// the 2s last-dimension weights (warp-uniform, one wavefront each) and RG
// values of V, and does RPL x 2s x RG FMAs.
template <typename T, int D, int S, int RC>
struct SpreadShape {
  static constexpr int TT = 2 * S;
  static constexpr int TTP = ttp_of(S);
  static constexpr int RG = (sizeof(T) == 4) ? ((RC % 8 == 0) ? 8 : ((RC % 4 == 0) ? 4 : 1))
                                             : ((RC % 4 == 0) ? 4 : ((RC % 2 == 0) ? 2 : 1));
  static constexpr int NG = RC / RG;
  static constexpr int RPL = (D == 3) ? 2 : 1;                 // grid rows per lane
  static constexpr int ROWS = (D == 1) ? 1 : ((D == 2) ? TT : TT * TT);
  static constexpr int LANES = ROWS / RPL * NG;
  static constexpr int THREADS = (LANES + 31) / 32 * 32;
  static constexpr int SUB = 32;                               // points per stage
  static constexpr int WPP = D * TTP;                          // window values per point
  static constexpr int VROW = (RC * sizeof(T) + 15) / 16 * 16 / sizeof(T);   // padded row
  static constexpr int STAGE = SUB * (WPP + VROW);             // elements per stage
  static constexpr size_t SMEM = 2 * STAGE * sizeof(T);
};

template <typename T, int D, int S, int RC>
__global__ void __launch_bounds__(SpreadShape<T, D, S, RC>::THREADS)
k_spread(const WinDev<T>* __restrict__ wins, const WinIO<T>* __restrict__ io,
         const int4* __restrict__ items, const T* __restrict__ V, int64_t ldv, int R) {
  using Sh = SpreadShape<T, D, S, RC>;
  constexpr int TT = Sh::TT, TTP = Sh::TTP, RG = Sh::RG, NG = Sh::NG, RPL = Sh::RPL;
  constexpr int SUB = Sh::SUB, WPP = Sh::WPP, VROW = Sh::VROW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);

  const int4 it = items[blockIdx.x];
  const WinDev<T> w = wins[it.x];
  if (io) {
    V = io[it.x].V;
    ldv = io[it.x].ldv;
  }
  const bool vec_ok = (ldv % (16 / (int)sizeof(T)) == 0) &&
                      ((reinterpret_cast<uintptr_t>(V) & 15) == 0);
  const int j0 = it.z, m = it.w;
  const int tid = threadIdx.x;
  const bool active = tid < Sh::LANES;
  const int g = active ? tid % NG : 0;
  const int rp = active ? tid / NG : 0;
  // rows of this lane: (t1, t2) and, for d = 3, (t1, t2 + s)
  const int t1 = (D == 3) ? rp / S : rp;
  const int t2 = (D == 3) ? rp % S : 0;
  const int col = g * RG;

  // stage loader: window values (contiguous) and V rows (gathered)
  auto stage = [&](int c, int buf) {
    T* ws = sm + buf * Sh::STAGE;
    T* vs = ws + SUB * WPP;
    const int q0 = c * SUB;
    const int ns = min(SUB, m - q0);
    constexpr int WCH = sizeof(T) * WPP / 16;              // 16-byte chunks per point
    const T* wsrc = w.wts + (int64_t)(j0 + q0) * WPP;
    for (int e = tid; e < ns * WCH; e += Sh::THREADS)
      cp_async16(ws + e * (16 / sizeof(T)), wsrc + e * (16 / sizeof(T)), 16);
    constexpr int VCH = sizeof(T) * VROW / 16;
    if (vec_ok) {
      for (int e = tid; e < ns * VCH; e += Sh::THREADS) {
        const int q = e / VCH, k = e - q * VCH;
        const int c0 = k * (16 / (int)sizeof(T));
        const int64_t i = __ldg(w.perm + j0 + q0 + q);
        const int valid = max(0, min(16 / (int)sizeof(T), R - c0));
        cp_async16(vs + q * VROW + c0, V + i * ldv + (valid > 0 ? c0 : 0), valid * (int)sizeof(T));
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

  T acc[RPL][TT][RG];
#pragma unroll
  for (int a = 0; a < RPL; ++a)
#pragma unroll
    for (int t = 0; t < TT; ++t)
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[a][t][q] = T(0);

  const int nchunk = (m + SUB - 1) / SUB;
  stage(0, 0);
  for (int c = 0; c < nchunk; ++c) {
    if (c + 1 < nchunk) {
      stage(c + 1, (c + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* ws = sm + (c & 1) * Sh::STAGE;
    const T* vs = ws + SUB * WPP;
    const int ns = min(SUB, m - c * SUB);
    for (int q = 0; q < ns; ++q) {
      const T* pw = ws + q * WPP;
      T wr[RPL];
      if constexpr (D == 3) {
        const T w1 = pw[t1];
        wr[0] = w1 * pw[TTP + t2];
        wr[1] = w1 * pw[TTP + t2 + S];
      } else if constexpr (D == 2) {
        wr[0] = pw[t1];
      } else {
        wr[0] = T(1);
      }
      T v[RG];
#pragma unroll
      for (int k = 0; k < RG; ++k) v[k] = vs[q * VROW + col + k];
      T a[RPL][RG];
#pragma unroll
      for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int k = 0; k < RG; ++k) a[r][k] = v[k] * wr[r];
      const T* wl = pw + (D - 1) * TTP;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const T wv = wl[t];
#pragma unroll
        for (int r = 0; r < RPL; ++r)
#pragma unroll
          for (int k = 0; k < RG; ++k) acc[r][t][k] = fma(a[r][k], wv, acc[r][t][k]);
      }
    }
    __syncthreads();   // the buffer of chunk c is refilled at iteration c + 1
  }
  if (!active || col >= R) return;   // padding lanes / padding columns
  int cc[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, cc);
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    int64_t base;
    if constexpr (D == 3) base = ((int64_t)(cc[0] + t1) * w.W + (cc[1] + t2 + r * S)) * w.W + cc[2];
    else if constexpr (D == 2) base = (int64_t)(cc[0] + t1) * w.W + cc[1];
    else base = cc[0];
    T* gp = w.grid + base * RC + col;
#pragma unroll
    for (int t = 0; t < TT; ++t) atomic_add_n<T, RG>(gp + (int64_t)t * RC, acc[r][t]);
  }
}

// ---------------------------------------------------------------------------
// Interpolation: Out[perm[j]][r] += scale * sum_a grid[a][r] prod_t psi_t(j, a_t - c_t)
// ---------------------------------------------------------------------------
// One CTA per (work item, slice of RS right-hand sides). The item's (2s)^d
// block is staged in shared memory once. Lane = (one right-hand side, PP
// points): the block values are read with 32-bit warp loads (the lanes of a
// point group read RS consecutive words, one wavefront) and each value feeds
// PP FMAs. The separable window is contracted one dimension at a time; the
// last-dimension weights of the lane's points stay in registers.
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
  static constexpr int WPP = D * TTP;
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

    T wl[PP][TT];
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int q = grp * PP + k;
#pragma unroll
      for (int t = 0; t < TT; ++t) wl[k][t] = (q < np) ? ws[q * WPS + (D - 1) * TTP + t] : T(0);
    }
    T acc[PP];
#pragma unroll
    for (int k = 0; k < PP; ++k) acc[k] = T(0);
    const T* hb = Hs + r;
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

// ---------------------------------------------------------------------------
// Dispatch over (d, s, RC)
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int RC>
cudaError_t spread_one(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                       int64_t n_items, const T* V, int64_t ldv, int R, cudaStream_t st) {
  using Sh = SpreadShape<T, D, S, RC>;
  if (n_items <= 0) return cudaSuccess;
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_spread<T, D, S, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_spread<T, D, S, RC><<<(unsigned)n_items, Sh::THREADS, Sh::SMEM, st>>>(wins, io, items, V, ldv, R);
  return cudaGetLastError();
}

template <typename T, int D, int S, int RC>
cudaError_t interp_one(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                       int64_t n_items, T* Out, int64_t ldo, int R, T scale, cudaStream_t st) {
  using Sh = InterpShape<T, D, S, RC>;
  if (n_items <= 0) return cudaSuccess;
  static bool attr_set = false;   // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_interp<T, D, S, RC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid((unsigned)n_items, (RC + Sh::RS - 1) / Sh::RS);
  k_interp<T, D, S, RC><<<grid, Sh::THREADS, Sh::SMEM, st>>>(wins, io, items, Out, ldo, R, scale);
  return cudaGetLastError();
}

#define AGP_S_SWITCH(FN, ...)                                   \
  switch (s) {                                                  \
    case 2: return FN<T, D, 2, RC>(__VA_ARGS__);                \
    case 3: return FN<T, D, 3, RC>(__VA_ARGS__);                \
    case 4: return FN<T, D, 4, RC>(__VA_ARGS__);                \
    case 5: return FN<T, D, 5, RC>(__VA_ARGS__);                \
    case 6: return FN<T, D, 6, RC>(__VA_ARGS__);                \
  }                                                             \
  return cudaErrorInvalidValue;

template <typename T, int D, int RC>
cudaError_t spread_s(int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                     int64_t n_items, const T* V, int64_t ldv, int R, cudaStream_t st) {
  AGP_S_SWITCH(spread_one, wins, io, items, n_items, V, ldv, R, st)
}

template <typename T, int D, int RC>
cudaError_t interp_s(int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                     int64_t n_items, T* Out, int64_t ldo, int R, T scale, cudaStream_t st) {
  AGP_S_SWITCH(interp_one, wins, io, items, n_items, Out, ldo, R, scale, st)
}

#define AGP_RC_SWITCH(FN, ...)                                          \
  if constexpr (sizeof(T) == 4) {                                       \
    if (RC == 32) return FN<T, D, 32>(__VA_ARGS__);                     \
    if (RC == 8) return FN<T, D, 8>(__VA_ARGS__);                       \
    if (RC == 1) return FN<T, D, 1>(__VA_ARGS__);                       \
  } else {                                                              \
    if (RC == 4) return FN<T, D, 4>(__VA_ARGS__);                       \
    if (RC == 1) return FN<T, D, 1>(__VA_ARGS__);                       \
  }                                                                     \
  return cudaErrorInvalidValue;

template <typename T, int D>
cudaError_t spread_rc(int RC, int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                      int64_t n_items, const T* V, int64_t ldv, int R, cudaStream_t st) {
  AGP_RC_SWITCH(spread_s, s, wins, io, items, n_items, V, ldv, R, st)
}

template <typename T, int D>
cudaError_t interp_rc(int RC, int s, const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                      int64_t n_items, T* Out, int64_t ldo, int R, T scale, cudaStream_t st) {
  AGP_RC_SWITCH(interp_s, s, wins, io, items, n_items, Out, ldo, R, scale, st)
}

}  // namespace

template <typename T>
cudaError_t spread_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, const T* V, int64_t ldv, int R,
                         cudaStream_t st) {
  if (d == 1) return spread_rc<T, 1>(RC, s, wins, io, items, n_items, V, ldv, R, st);
  if (d == 2) return spread_rc<T, 2>(RC, s, wins, io, items, n_items, V, ldv, R, st);
  if (d == 3) return spread_rc<T, 3>(RC, s, wins, io, items, n_items, V, ldv, R, st);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t interp_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, T* Out, int64_t ldo, int R,
                         T scale, cudaStream_t st) {
  if (d == 1) return interp_rc<T, 1>(RC, s, wins, io, items, n_items, Out, ldo, R, scale, st);
  if (d == 2) return interp_rc<T, 2>(RC, s, wins, io, items, n_items, Out, ldo, R, scale, st);
  if (d == 3) return interp_rc<T, 3>(RC, s, wins, io, items, n_items, Out, ldo, R, scale, st);
  return cudaErrorInvalidValue;
}

template cudaError_t spread_items<float>(const WinDev<float>*, const WinIO<float>*, const int4*,
                                         int64_t, int, int, int, const float*, int64_t, int,
                                         cudaStream_t);
template cudaError_t spread_items<double>(const WinDev<double>*, const WinIO<double>*, const int4*,
                                          int64_t, int, int, int, const double*, int64_t, int,
                                          cudaStream_t);
template cudaError_t interp_items<float>(const WinDev<float>*, const WinIO<float>*, const int4*,
                                         int64_t, int, int, int, float*, int64_t, int, float,
                                         cudaStream_t);
template cudaError_t interp_items<double>(const WinDev<double>*, const WinIO<double>*, const int4*,
                                          int64_t, int, int, int, double*, int64_t, int, double,
                                          cudaStream_t);

}  // namespace agp
