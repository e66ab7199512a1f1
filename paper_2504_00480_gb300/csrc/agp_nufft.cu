// Spreading (adjoint NFFT, Appendix A step 3 transposed) and interpolation
// (NFFT, Appendix A step 3) of the additive-kernel fast summation, Sec. 3.1
// eq. (3.3).
//
// Work is split into items: one item = up to kItemPoints points that share a
// grid cell (points are sorted by cell at plan time). All points of an item
// touch the same (2s)^d block of grid points, so
//  * spreading accumulates the whole block for the item in REGISTERS (one
//    CTA, thread = one grid row of 2s points x RG right-hand sides) and adds
//    it to the grid once per item with vector atomics;
//  * interpolation stages the block once per item in SHARED MEMORY and every
//    thread evaluates PP points x RG right-hand sides from it, contracting the
//    separable window dimension by dimension.
// Every window and right-hand side of one dimension d runs in one launch.
#include "agp_internal.cuh"

namespace agp {
namespace {

template <typename T, int RC>
struct RGOf {
  static constexpr int v = (sizeof(T) == 4) ? ((RC % 4 == 0) ? 4 : 1) : ((RC % 2 == 0) ? 2 : 1);
};

template <typename T, int RG>
__device__ __forceinline__ void atomic_add_n(T* p, const T* a) {
  if constexpr (sizeof(T) == 4 && RG == 4) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(a[0], a[1], a[2], a[3]));
  } else {
#pragma unroll
    for (int i = 0; i < RG; ++i) atomicAdd(p + i, a[i]);
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

// ---------------------------------------------------------------------------
// Spreading: grid[a][r] += sum_j V[perm[j]][r] prod_t psi(u_jt - l_t)
// ---------------------------------------------------------------------------
constexpr int groups_per_block(int ng, int rows) {
  int b = ng;
  while (b > 1 && rows * b > 1024) b /= 2;
  return b;
}

template <typename T, int D, int S, int RC>
struct SpreadShape {
  static constexpr int TT = 2 * S;                 // taps per dimension
  static constexpr int RG = RGOf<T, RC>::v;        // right-hand sides per thread
  static constexpr int NG = RC / RG;               // right-hand-side groups
  static constexpr int ROWS = (D == 1) ? 1 : ((D == 2) ? TT : TT * TT);
  static constexpr int NGB = groups_per_block(NG, ROWS);   // groups per CTA
  static constexpr int GY = NG / NGB;                      // CTAs per item (blockIdx.y)
  static constexpr int THREADS = ROWS * NGB;
  static constexpr int SUB = 32;                   // points staged per pass
  static constexpr int WPP = D * TT;               // window values per point
};

template <typename T, int D, int S, int RC>
__global__ void __launch_bounds__(SpreadShape<T, D, S, RC>::THREADS)
k_spread(const WinDev<T>* __restrict__ wins, const int4* __restrict__ items,
         const T* __restrict__ V, int64_t ldv, int R, T kb_b, T kb_norm) {
  using Sh = SpreadShape<T, D, S, RC>;
  constexpr int TT = Sh::TT, RG = Sh::RG, NGB = Sh::NGB, SUB = Sh::SUB, WPP = Sh::WPP;
  __shared__ T ws[SUB * WPP];
  __shared__ __align__(16) T vs[SUB * RC];

  const int4 it = items[blockIdx.x];
  const WinDev<T> w = wins[it.x];
  const int j0 = it.z, m = it.w;
  int c[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, c);

  const int tid = threadIdx.x;
  const int g = blockIdx.y * NGB + tid % NGB;
  const int row = tid / NGB;
  const int t1 = (D == 3) ? row / TT : row;
  const int t2 = (D == 3) ? row % TT : 0;

  T acc[TT][RG];
#pragma unroll
  for (int t = 0; t < TT; ++t)
#pragma unroll
    for (int q = 0; q < RG; ++q) acc[t][q] = T(0);

  const T sf = T(S);
  const T nos = T(w.n_os);
  for (int sub = 0; sub < m; sub += SUB) {
    const int ns = min(SUB, m - sub);
    for (int e = tid; e < ns * WPP; e += Sh::THREADS) {
      const int q = e / WPP, rem = e - q * WPP, dim = rem / TT, t = rem - dim * TT;
      const T u = w.xs[(int64_t)dim * w.n + j0 + sub + q] * nos;
      const T frac = u - dev_floor(u);
      ws[e] = kb_psi(frac + T(S - 1 - t), sf, kb_b, kb_norm);
    }
    for (int e = tid; e < ns * RC; e += Sh::THREADS) {
      const int q = e / RC, r = e - q * RC;
      const int64_t i = w.perm[j0 + sub + q];
      vs[e] = (r < R) ? V[i * ldv + r] : T(0);
    }
    __syncthreads();
    for (int q = 0; q < ns; ++q) {
      const T* wq = ws + q * WPP;
      T wrow;
      if constexpr (D == 3) wrow = wq[t1] * wq[TT + t2];
      else if constexpr (D == 2) wrow = wq[t1];
      else wrow = T(1);
      T a[RG];
#pragma unroll
      for (int k = 0; k < RG; ++k) a[k] = vs[q * RC + g * RG + k] * wrow;
      const T* wl = wq + (D - 1) * TT;
#pragma unroll
      for (int t = 0; t < TT; ++t) {
        const T wv = wl[t];
#pragma unroll
        for (int k = 0; k < RG; ++k) acc[t][k] = fma(a[k], wv, acc[t][k]);
      }
    }
    __syncthreads();
  }
  if (g * RG >= R) return;   // these columns are padding: nothing to add
  int64_t base;
  if constexpr (D == 3) base = ((int64_t)(c[0] + t1) * w.W + (c[1] + t2)) * w.W + c[2];
  else if constexpr (D == 2) base = (int64_t)(c[0] + t1) * w.W + c[1];
  else base = c[0];
  T* gp = w.grid + base * RC + g * RG;
#pragma unroll
  for (int t = 0; t < TT; ++t) atomic_add_n<T, RG>(gp + (int64_t)t * RC, acc[t]);
}

// ---------------------------------------------------------------------------
// Interpolation: Out[perm[j]][r] += scale * sum_a grid[a][r] prod_t psi(u_jt - l_t)
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int RC>
struct InterpShape {
  static constexpr int TT = 2 * S;
  static constexpr int RS = (RC > 16) ? 16 : RC;   // right-hand sides per CTA (blockIdx.y slices)
  static constexpr int RG = RGOf<T, RS>::v;
  static constexpr int NGS = RS / RG;
  static constexpr int THREADS = 128;
  static constexpr int NSLOT = THREADS / NGS;      // point slots per CTA
  static constexpr int PP = 2;                     // points per thread
  static constexpr int PTS = NSLOT * PP;           // points per pass
  static constexpr int BLK = (D == 1) ? TT : ((D == 2) ? TT * TT : TT * TT * TT);
  static constexpr int WPP = D * TT;
  static constexpr size_t SMEM = sizeof(T) * ((size_t)BLK * RS + (size_t)PTS * WPP);
};

template <typename T, int D, int S, int RC>
__global__ void __launch_bounds__(128)
k_interp(const WinDev<T>* __restrict__ wins, const int4* __restrict__ items,
         T* __restrict__ Out, int64_t ldo, int R, T scale, T kb_b, T kb_norm, int vec_ok) {
  using Sh = InterpShape<T, D, S, RC>;
  constexpr int TT = Sh::TT, RS = Sh::RS, RG = Sh::RG, NGS = Sh::NGS, PP = Sh::PP;
  constexpr int NSLOT = Sh::NSLOT, PTS = Sh::PTS, BLK = Sh::BLK, WPP = Sh::WPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Hs = reinterpret_cast<T*>(smem_raw);   // [BLK][RS]
  T* wsm = Hs + BLK * RS;                    // [PTS][WPP]

  const int rs0 = blockIdx.y * RS;
  if (rs0 >= R) return;
  const int4 it = items[blockIdx.x];
  const WinDev<T> w = wins[it.x];
  const int j0 = it.z, m = it.w;
  int c[3] = {0, 0, 0};
  decode_cell<D>(it.y, w.N, c);
  const int tid = threadIdx.x;

  // Stage the item's (2s)^d block, columns rs0 .. rs0+RS-1.
  for (int e = tid; e < BLK * RS; e += Sh::THREADS) {
    const int ci = e / RS, r = e - ci * RS;
    int64_t gi;
    if constexpr (D == 3) {
      const int a3 = ci % TT, a2 = (ci / TT) % TT, a1 = ci / (TT * TT);
      gi = ((int64_t)(c[0] + a1) * w.W + (c[1] + a2)) * w.W + (c[2] + a3);
    } else if constexpr (D == 2) {
      const int a2 = ci % TT, a1 = ci / TT;
      gi = (int64_t)(c[0] + a1) * w.W + (c[1] + a2);
    } else {
      gi = c[0] + ci;
    }
    Hs[e] = w.grid[gi * RC + rs0 + r];
  }

  const int g = tid % NGS;
  const int slot = tid / NGS;
  const T sf = T(S);
  const T nos = T(w.n_os);
  for (int p0 = 0; p0 < m; p0 += PTS) {
    const int np = min(PTS, m - p0);
    __syncthreads();   // previous pass done with wsm (and the block is staged)
    for (int e = tid; e < np * WPP; e += Sh::THREADS) {
      const int q = e / WPP, rem = e - q * WPP, dim = rem / TT, t = rem - dim * TT;
      const T u = w.xs[(int64_t)dim * w.n + j0 + p0 + q] * nos;
      const T frac = u - dev_floor(u);
      wsm[e] = kb_psi(frac + T(S - 1 - t), sf, kb_b, kb_norm);
    }
    __syncthreads();

    int qs[PP];
    T wl[PP][TT];
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      qs[k] = slot + k * NSLOT;
      const bool ok = qs[k] < np;
#pragma unroll
      for (int t = 0; t < TT; ++t) wl[k][t] = ok ? wsm[qs[k] * WPP + (D - 1) * TT + t] : T(0);
    }
    T acc[PP][RG];
#pragma unroll
    for (int k = 0; k < PP; ++k)
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[k][q] = T(0);

    const T* hb = Hs + g * RG;
    if constexpr (D == 1) {
#pragma unroll
      for (int t3 = 0; t3 < TT; ++t3) {
        T h[RG];
#pragma unroll
        for (int q = 0; q < RG; ++q) h[q] = hb[t3 * RS + q];
#pragma unroll
        for (int k = 0; k < PP; ++k)
#pragma unroll
          for (int q = 0; q < RG; ++q) acc[k][q] = fma(wl[k][t3], h[q], acc[k][q]);
      }
    } else {
      constexpr int N1 = (D == 3) ? TT : 1;
      for (int t1 = 0; t1 < N1; ++t1) {
        T u1[PP][RG];
#pragma unroll
        for (int k = 0; k < PP; ++k)
#pragma unroll
          for (int q = 0; q < RG; ++q) u1[k][q] = T(0);
        for (int t2 = 0; t2 < TT; ++t2) {
          T u2[PP][RG];
#pragma unroll
          for (int k = 0; k < PP; ++k)
#pragma unroll
            for (int q = 0; q < RG; ++q) u2[k][q] = T(0);
          const T* hrow = hb + ((t1 * TT + t2) * TT) * RS;
#pragma unroll
          for (int t3 = 0; t3 < TT; ++t3) {
            T h[RG];
#pragma unroll
            for (int q = 0; q < RG; ++q) h[q] = hrow[t3 * RS + q];
#pragma unroll
            for (int k = 0; k < PP; ++k)
#pragma unroll
              for (int q = 0; q < RG; ++q) u2[k][q] = fma(wl[k][t3], h[q], u2[k][q]);
          }
          // weight of tap t2 along the second-to-last dimension
#pragma unroll
          for (int k = 0; k < PP; ++k) {
            const T w2 = (qs[k] < np) ? wsm[qs[k] * WPP + (D - 2) * TT + t2] : T(0);
#pragma unroll
            for (int q = 0; q < RG; ++q) u1[k][q] = fma(w2, u2[k][q], u1[k][q]);
          }
        }
        if constexpr (D == 3) {
#pragma unroll
          for (int k = 0; k < PP; ++k) {
            const T w1 = (qs[k] < np) ? wsm[qs[k] * WPP + t1] : T(0);
#pragma unroll
            for (int q = 0; q < RG; ++q) acc[k][q] = fma(w1, u1[k][q], acc[k][q]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < PP; ++k)
#pragma unroll
            for (int q = 0; q < RG; ++q) acc[k][q] = u1[k][q];
        }
      }
    }

#pragma unroll
    for (int k = 0; k < PP; ++k) {
      if (qs[k] >= np) continue;
      const int64_t i = w.perm[j0 + p0 + qs[k]];
      const int col = rs0 + g * RG;
      T* op = Out + i * ldo + col;
      T v[RG];
#pragma unroll
      for (int q = 0; q < RG; ++q) v[q] = scale * acc[k][q];
      if (vec_ok && col + RG <= R) {
        atomic_add_n<T, RG>(op, v);
      } else {
#pragma unroll
        for (int q = 0; q < RG; ++q)
          if (col + q < R) atomicAdd(op + q, v[q]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Dispatch over (d, s, RC)
// ---------------------------------------------------------------------------
template <typename T, int D, int S, int RC>
cudaError_t spread_one(const WinDev<T>* wins, const int4* items, int64_t n_items, const T* V,
                       int64_t ldv, int R, T b, T norm, cudaStream_t st) {
  using Sh = SpreadShape<T, D, S, RC>;
  if (n_items <= 0) return cudaSuccess;
  dim3 grid((unsigned)n_items, Sh::GY);
  k_spread<T, D, S, RC><<<grid, Sh::THREADS, 0, st>>>(wins, items, V, ldv, R, b, norm);
  return cudaGetLastError();
}

template <typename T, int D, int S, int RC>
cudaError_t interp_one(const WinDev<T>* wins, const int4* items, int64_t n_items, T* Out,
                       int64_t ldo, int R, T scale, T b, T norm, int vec_ok, cudaStream_t st) {
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
  k_interp<T, D, S, RC><<<grid, Sh::THREADS, Sh::SMEM, st>>>(wins, items, Out, ldo, R, scale, b,
                                                           norm, vec_ok);
  return cudaGetLastError();
}

template <typename T, int D, int RC>
cudaError_t spread_s(int s, const WinDev<T>* wins, const int4* items, int64_t n_items,
                     const T* V, int64_t ldv, int R, T b, T norm, cudaStream_t st) {
  switch (s) {
    case 2: return spread_one<T, D, 2, RC>(wins, items, n_items, V, ldv, R, b, norm, st);
    case 3: return spread_one<T, D, 3, RC>(wins, items, n_items, V, ldv, R, b, norm, st);
    case 4: return spread_one<T, D, 4, RC>(wins, items, n_items, V, ldv, R, b, norm, st);
    case 5: return spread_one<T, D, 5, RC>(wins, items, n_items, V, ldv, R, b, norm, st);
    case 6: return spread_one<T, D, 6, RC>(wins, items, n_items, V, ldv, R, b, norm, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int D, int RC>
cudaError_t interp_s(int s, const WinDev<T>* wins, const int4* items, int64_t n_items, T* Out,
                     int64_t ldo, int R, T scale, T b, T norm, int vec_ok, cudaStream_t st) {
  switch (s) {
    case 2: return interp_one<T, D, 2, RC>(wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    case 3: return interp_one<T, D, 3, RC>(wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    case 4: return interp_one<T, D, 4, RC>(wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    case 5: return interp_one<T, D, 5, RC>(wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    case 6: return interp_one<T, D, 6, RC>(wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int D>
cudaError_t spread_rc(int RC, int s, const WinDev<T>* wins, const int4* items, int64_t n_items,
                      const T* V, int64_t ldv, int R, T b, T norm, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (RC == 32) return spread_s<T, D, 32>(s, wins, items, n_items, V, ldv, R, b, norm, st);
    if (RC == 8) return spread_s<T, D, 8>(s, wins, items, n_items, V, ldv, R, b, norm, st);
    if (RC == 1) return spread_s<T, D, 1>(s, wins, items, n_items, V, ldv, R, b, norm, st);
  } else {
    if (RC == 4) return spread_s<T, D, 4>(s, wins, items, n_items, V, ldv, R, b, norm, st);
    if (RC == 1) return spread_s<T, D, 1>(s, wins, items, n_items, V, ldv, R, b, norm, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int D>
cudaError_t interp_rc(int RC, int s, const WinDev<T>* wins, const int4* items, int64_t n_items,
                      T* Out, int64_t ldo, int R, T scale, T b, T norm, int vec_ok,
                      cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (RC == 32) return interp_s<T, D, 32>(s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    if (RC == 8) return interp_s<T, D, 8>(s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    if (RC == 1) return interp_s<T, D, 1>(s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  } else {
    if (RC == 4) return interp_s<T, D, 4>(s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
    if (RC == 1) return interp_s<T, D, 1>(s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t spread_d(int d, int RC, int s, const WinDev<T>* wins, const int4* items,
                     int64_t n_items, const T* V, int64_t ldv, int R, T b, T norm,
                     cudaStream_t st) {
  if (d == 1) return spread_rc<T, 1>(RC, s, wins, items, n_items, V, ldv, R, b, norm, st);
  if (d == 2) return spread_rc<T, 2>(RC, s, wins, items, n_items, V, ldv, R, b, norm, st);
  if (d == 3) return spread_rc<T, 3>(RC, s, wins, items, n_items, V, ldv, R, b, norm, st);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t interp_d(int d, int RC, int s, const WinDev<T>* wins, const int4* items,
                     int64_t n_items, T* Out, int64_t ldo, int R, T scale, T b, T norm,
                     cudaStream_t st) {
  const int vec_ok = (ldo % 4 == 0) && ((reinterpret_cast<uintptr_t>(Out) & 15) == 0);
  if (d == 1) return interp_rc<T, 1>(RC, s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  if (d == 2) return interp_rc<T, 2>(RC, s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  if (d == 3) return interp_rc<T, 3>(RC, s, wins, items, n_items, Out, ldo, R, scale, b, norm, vec_ok, st);
  return cudaErrorInvalidValue;
}

}  // namespace

template <typename T>
cudaError_t launch_spread(const agp_plan_s* plan, int d, int RC, const T* V, int64_t ldv, int R,
                          cudaStream_t st) {
  const int64_t a = plan->items_by_d[d - 1], b = plan->items_by_d[d];
  return spread_d<T>(d, RC, plan->s, reinterpret_cast<const WinDev<T>*>(plan->wins_dev),
                     plan->items_all + a, b - a, V, ldv, R, (T)plan->kb_b, (T)plan->kb_norm, st);
}

template <typename T>
cudaError_t launch_interp(const agp_plan_s* plan, int d, int RC, T* Out, int64_t ldo, int R,
                          T scale, cudaStream_t st) {
  const int64_t a = plan->items_by_d[d - 1], b = plan->items_by_d[d];
  return interp_d<T>(d, RC, plan->s, reinterpret_cast<const WinDev<T>*>(plan->wins_dev),
                     plan->items_all + a, b - a, Out, ldo, R, scale, (T)plan->kb_b,
                     (T)plan->kb_norm, st);
}

template <typename T>
cudaError_t launch_spread_window(const agp_plan_s* plan, int wi, int RC, const T* V, int64_t ldv,
                                 int R, cudaStream_t st) {
  const Window& w = plan->win[wi];
  return spread_d<T>(w.d, RC, plan->s, reinterpret_cast<const WinDev<T>*>(plan->wins_dev),
                     w.items, w.n_items, V, ldv, R, (T)plan->kb_b, (T)plan->kb_norm, st);
}

template <typename T>
cudaError_t launch_interp_window(const agp_plan_s* plan, int wi, int RC, T* Out, int64_t ldo,
                                 int R, T scale, cudaStream_t st) {
  const Window& w = plan->win[wi];
  return interp_d<T>(w.d, RC, plan->s, reinterpret_cast<const WinDev<T>*>(plan->wins_dev),
                     w.items, w.n_items, Out, ldo, R, scale, (T)plan->kb_b, (T)plan->kb_norm, st);
}

template cudaError_t launch_spread<float>(const agp_plan_s*, int, int, const float*, int64_t, int, cudaStream_t);
template cudaError_t launch_spread<double>(const agp_plan_s*, int, int, const double*, int64_t, int, cudaStream_t);
template cudaError_t launch_interp<float>(const agp_plan_s*, int, int, float*, int64_t, int, float, cudaStream_t);
template cudaError_t launch_interp<double>(const agp_plan_s*, int, int, double*, int64_t, int, double, cudaStream_t);
template cudaError_t launch_spread_window<float>(const agp_plan_s*, int, int, const float*, int64_t, int, cudaStream_t);
template cudaError_t launch_spread_window<double>(const agp_plan_s*, int, int, const double*, int64_t, int, cudaStream_t);
template cudaError_t launch_interp_window<float>(const agp_plan_s*, int, int, float*, int64_t, int, float, cudaStream_t);
template cudaError_t launch_interp_window<double>(const agp_plan_s*, int, int, double*, int64_t, int, double, cudaStream_t);

}  // namespace agp
