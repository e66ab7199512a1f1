// The DFT stage of one application (Appendix A steps 2 and 4 around the
// spectral multiply of Sec. 3.1 eq. (3.3)) for every d = 2 and d = 3 window of
// a plan or batch in three launches, whatever the number of window groups:
//
//   F1  per grid plane (d = 3: fixed a0) or row (d = 2): the forward pruned
//       DFT along the last axis (real -> Hermitian half) and, for d = 3, along
//       the middle axis, in shared memory; writes the plane of the spectrum
//       [a0][k1][k2][r] (d = 2: [a0][k1][r]) to specA.
//   F2  per column of the first axis: the forward DFT along a0, the multiply
//       by the deconvolved coefficients D_k of the kernel (or of its
//       ell-derivative), and the inverse DFT back to a0, in shared memory and
//       in place in specA.
//   F3  per grid plane or row: the inverse DFTs of F1 in reverse order,
//       writing the grid.
//
// The transforms are the pruned dense DFTs of agp_fft.cu (grid points a in
// the active box [0, W), frequencies k in [-N/2, N/2], the last axis real <->
// half spectrum k in [0, N/2]) with the same twiddle table; they differ only
// in the order of the summations (each output sums over the same inputs in
// the same order). Keeping a plane's transforms along two axes in shared
// memory, and the first axis's forward transform, multiply and inverse in one
// pass, replaces seven launches per d = 3 group (five per d = 2 group) and
// the spectrum's round trips through L2 between them.
//
// One launch serves all groups: each CTA finds its task (group) from its
// index in a small table passed by value.
#include <algorithm>

#include "agp_internal.cuh"

namespace agp {
namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

constexpr int kDftMaxTasks = 8;
constexpr int kDftThreads = 256;
constexpr int kDftCB = 32;            // columns per CTA of F2
constexpr size_t kDftSmemCap = 100 * 1024;   // two CTAs per SM

struct DftTask {
  const FftWin* tab;      // the group's windows
  int count, d, N, W, K, KH;
  int RB;                 // grid columns per CTA of F1 / F3
  int per_win;            // CTAs per window of this launch
  int begin;              // first CTA of the task
};

struct DftTasks {
  DftTask t[kDftMaxTasks];
  int n;
  int RC;                 // grid columns of the pass
  int der;                // 0: kernel coefficients, 1: ell-derivative
};

// the task of CTA `bx`, the window and the CTA's index within the window
// (false: none); static indices only, so the table stays in parameter space
__device__ __forceinline__ bool dft_task(const DftTasks& ts, int bx, DftTask& t, int& win,
                                         int& local) {
  int sel = -1;
#pragma unroll
  for (int q = 0; q < kDftMaxTasks; ++q)
    if (q < ts.n && bx >= ts.t[q].begin && bx < ts.t[q].begin + ts.t[q].count * ts.t[q].per_win)
      sel = q;
  if (sel < 0) return false;
#pragma unroll
  for (int q = 0; q < kDftMaxTasks; ++q)
    if (q == sel) t = ts.t[q];
  win = (bx - t.begin) / t.per_win;
  local = (bx - t.begin) - win * t.per_win;
  return true;
}

// ---------------------------------------------------------------------------
// Register-tiled transforms along one axis of a shared-memory block. A
// thread computes KQ outputs (consecutive frequencies or grid points) for JQ
// consecutive columns, so every input value it loads feeds KQ outputs and
// every twiddle JQ of them; each output still sums its inputs in ascending
// order, one FMA at a time.
// ---------------------------------------------------------------------------
constexpr int kDftKQ = 4;

// Column j of a block of JB-wide rows RS apart starts at (j / JB) RS + j % JB.
__device__ __forceinline__ int dft_col(int j, int JB, int RS) { return (j / JB) * RS + j % JB; }

// forward, real input: out(k, j) = sum_m in[m SM + col(j)] w(k, m), w(k, m) =
// tw[k W + m] (k < KO; rows clamped to KO - 1 past the end, not stored)
template <typename T, int JQ, typename Store>
__device__ __forceinline__ void dft_fwd_real(const T* in, int M, int SM, int J, int JB, int RS,
                                             int KO, const typename Cx<T>::t* tw, int W,
                                             Store store) {
  using T2 = typename Cx<T>::t;
  const int nk = (KO + kDftKQ - 1) / kDftKQ, nj = (J + JQ - 1) / JQ;
  for (int e = threadIdx.x; e < nk * nj; e += blockDim.x) {
    const int j0 = (e % nj) * JQ, k0 = (e / nj) * kDftKQ;
    T re[kDftKQ][JQ], im[kDftKQ][JQ];
    const T2* tk[kDftKQ];
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q) {
      tk[q] = tw + (int64_t)min(k0 + q, KO - 1) * W;
#pragma unroll
      for (int c = 0; c < JQ; ++c) re[q][c] = im[q][c] = T(0);
    }
    int off[JQ];
#pragma unroll
    for (int c = 0; c < JQ; ++c) off[c] = dft_col(min(j0 + c, J - 1), JB, RS);
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
      T x[JQ];
#pragma unroll
      for (int c = 0; c < JQ; ++c) x[c] = (j0 + c < J) ? in[m * SM + off[c]] : T(0);
#pragma unroll
      for (int q = 0; q < kDftKQ; ++q) {
        const T2 w = __ldg(tk[q] + m);
#pragma unroll
        for (int c = 0; c < JQ; ++c) {
          re[q][c] = fma(x[c], w.x, re[q][c]);
          im[q][c] = fma(x[c], w.y, im[q][c]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q)
#pragma unroll
      for (int c = 0; c < JQ; ++c)
        if (k0 + q < KO && j0 + c < J) {
          T2 v;
          v.x = re[q][c];
          v.y = im[q][c];
          store(k0 + q, j0 + c, v);
        }
  }
}

// complex input: forward out(k, j) = sum_m in[m SM + j] w(k, m) (conj = false),
// inverse out(k, j) = sum_m in[m SM + j] conj(w(m, k)) (conj = true; k a grid
// point, m a frequency)
template <typename T, int JQ, bool CONJ, typename Store>
__device__ __forceinline__ void dft_cplx(const typename Cx<T>::t* in, int M, int SM, int J,
                                         int KO, const typename Cx<T>::t* tw, int W,
                                         Store store) {
  using T2 = typename Cx<T>::t;
  const int nk = (KO + kDftKQ - 1) / kDftKQ, nj = (J + JQ - 1) / JQ;
  for (int e = threadIdx.x; e < nk * nj; e += blockDim.x) {
    const int j0 = (e % nj) * JQ, k0 = (e / nj) * kDftKQ;
    T re[kDftKQ][JQ], im[kDftKQ][JQ];
    int kc[kDftKQ];
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q) {
      kc[q] = min(k0 + q, KO - 1);
#pragma unroll
      for (int c = 0; c < JQ; ++c) re[q][c] = im[q][c] = T(0);
    }
#pragma unroll 4
    for (int m = 0; m < M; ++m) {
      T2 x[JQ];
#pragma unroll
      for (int c = 0; c < JQ; ++c) {
        if (j0 + c < J) {
          x[c] = in[m * SM + j0 + c];
        } else {
          x[c].x = T(0);
          x[c].y = T(0);
        }
      }
#pragma unroll
      for (int q = 0; q < kDftKQ; ++q) {
        const T2 w = __ldg(tw + (CONJ ? (int64_t)m * W + kc[q] : (int64_t)kc[q] * W + m));
#pragma unroll
        for (int c = 0; c < JQ; ++c) {
          if (CONJ) {            // x conj(w)
            re[q][c] = fma(x[c].x, w.x, re[q][c]);
            re[q][c] = fma(x[c].y, w.y, re[q][c]);
            im[q][c] = fma(x[c].y, w.x, im[q][c]);
            im[q][c] = fma(-x[c].x, w.y, im[q][c]);
          } else {               // x w
            re[q][c] = fma(x[c].x, w.x, re[q][c]);
            re[q][c] = fma(-x[c].y, w.y, re[q][c]);
            im[q][c] = fma(x[c].x, w.y, im[q][c]);
            im[q][c] = fma(x[c].y, w.x, im[q][c]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q)
#pragma unroll
      for (int c = 0; c < JQ; ++c)
        if (k0 + q < KO && j0 + c < J) {
          T2 v;
          v.x = re[q][c];
          v.y = im[q][c];
          store(k0 + q, j0 + c, v);
        }
  }
}

// Hermitian half -> real: out(a, j) = sum_k s_k Re(in[k SM + col(j)] conj(w(k, a))),
// s_0 = 1, s_k = 2 (k >= 1), w(k, a) = twh[k W + a]
template <typename T, int JQ, typename Store>
__device__ __forceinline__ void dft_half_real(const typename Cx<T>::t* in, int KH, int SM, int J,
                                              int JB, int RS, int AO,
                                              const typename Cx<T>::t* twh, int W,
                                              Store store) {
  using T2 = typename Cx<T>::t;
  const int na = (AO + kDftKQ - 1) / kDftKQ, nj = (J + JQ - 1) / JQ;
  for (int e = threadIdx.x; e < na * nj; e += blockDim.x) {
    const int j0 = (e % nj) * JQ, a0 = (e / nj) * kDftKQ;
    T acc[kDftKQ][JQ];
    int ac[kDftKQ];
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q) {
      ac[q] = min(a0 + q, AO - 1);
#pragma unroll
      for (int c = 0; c < JQ; ++c) acc[q][c] = T(0);
    }
    int off[JQ];
#pragma unroll
    for (int c = 0; c < JQ; ++c) off[c] = dft_col(min(j0 + c, J - 1), JB, RS);
#pragma unroll 4
    for (int k = 0; k < KH; ++k) {
      const T sk = (k == 0) ? T(1) : T(2);
      T2 x[JQ];
#pragma unroll
      for (int c = 0; c < JQ; ++c) {
        if (j0 + c < J) {
          x[c] = in[k * SM + off[c]];
        } else {
          x[c].x = T(0);
          x[c].y = T(0);
        }
      }
#pragma unroll
      for (int q = 0; q < kDftKQ; ++q) {
        const T2 w = __ldg(twh + (int64_t)k * W + ac[q]);
#pragma unroll
        for (int c = 0; c < JQ; ++c) {
          acc[q][c] = fma(sk * x[c].x, w.x, acc[q][c]);
          acc[q][c] = fma(sk * x[c].y, w.y, acc[q][c]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kDftKQ; ++q)
#pragma unroll
      for (int c = 0; c < JQ; ++c)
        if (a0 + q < AO && j0 + c < J) store(a0 + q, j0 + c, acc[q][c]);
  }
}

// ---------------------------------------------------------------------------
// F1: forward along the last axis (and the middle axis for d = 3) of one plane
// ---------------------------------------------------------------------------
// Shared memory (T): G[W(a1)][W(a2)][RB] for d = 3 (d = 2: G[W(a1)][RB]),
// then S1[W(a1)][KH][RB] complex (d = 3 only).
template <typename T>
__global__ void __launch_bounds__(kDftThreads) k_dft_f1(const DftTasks ts) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char dft_smem[];
  int win, local;
  DftTask t;
  if (!dft_task(ts, blockIdx.x, t, win, local)) return;
  const FftWin f = t.tab[win];
  const int RC = ts.RC, RB = t.RB, W = t.W, K = t.K, KH = t.KH;
  const int nrc = RC / RB;
  const int a0 = local / nrc, r0 = (local - a0 * nrc) * RB;
  const T2* tw = reinterpret_cast<const T2*>(f.tw);
  const T2* twh = tw + (int64_t)(KH - 1) * W;        // row of k = 0
  const T* grid = reinterpret_cast<const T*>(f.grid);
  T2* spec = reinterpret_cast<T2*>(f.specA);
  T* G = reinterpret_cast<T*>(dft_smem);
  const int rows = t.d == 3 ? W : 1;                  // a1 rows of the plane
  // the plane (row) of the grid, columns r0 .. r0 + RB - 1
  const T* src = grid + (int64_t)a0 * rows * W * RC + r0;
  for (int e = threadIdx.x; e < rows * W * RB; e += blockDim.x) {
    const int rb = e % RB, p = e / RB;              // p = a1 W + a2
    G[e] = src[(int64_t)p * RC + rb];
  }
  __syncthreads();
  if (t.d == 2) {
    // spec[a0][k][r] = sum_a G[a][r] w(k, a), k in [0, N/2]
    T2* dst = spec + (int64_t)a0 * KH * RC + r0;
    dft_fwd_real<T, 2>(G, W, RB, RB, RB, 0, KH, twh, W,
                       [&](int k, int j, T2 v) { dst[(int64_t)k * RC + j] = v; });
    return;
  }
  // d = 3: last axis of every row a1 (columns j = a1 RB + rb), S1[a1][k2][rb]
  T2* S1 = reinterpret_cast<T2*>(dft_smem + (((size_t)W * W * RB * sizeof(T) + 15) / 16) * 16);
  dft_fwd_real<T, 2>(G, W, RB, W * RB, RB, W * RB, KH, twh, W, [&](int k, int j, T2 v) {
    const int a1 = j / RB, rb = j - a1 * RB;
    S1[((int64_t)a1 * KH + k) * RB + rb] = v;
  });
  __syncthreads();
  // middle axis: spec[a0][k1][k2][r] = sum_a1 S1[a1][k2][r] w(k1, a1); columns
  // j = k2 RB + rb
  T2* dst = spec + (int64_t)a0 * K * KH * RC + r0;
  dft_cplx<T, 2, false>(S1, W, KH * RB, KH * RB, K, tw, W, [&](int k1, int j, T2 v) {
    const int k2 = j / RB, rb = j - k2 * RB;
    dst[((int64_t)k1 * KH + k2) * RC + rb] = v;
  });
}

// ---------------------------------------------------------------------------
// F2: forward along a0, multiply by D_k, inverse along a0 (in place in specA)
// ---------------------------------------------------------------------------
// Columns c = (k1 KH + k2) RC + r (d = 3; d = 2: c = k1 RC + r), C = P2 RC of
// them, P2 = K KH (d = 3) or KH (d = 2); column c of plane a0 at
// specA[a0 C + c]. Shared memory: X[W][kDftCB], Y[K][kDftCB] complex.
template <typename T>
__global__ void __launch_bounds__(kDftThreads) k_dft_f2(const DftTasks ts) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char dft_smem[];
  int win, local;
  DftTask t;
  if (!dft_task(ts, blockIdx.x, t, win, local)) return;
  const FftWin f = t.tab[win];
  const int RC = ts.RC, W = t.W, K = t.K;
  const int64_t P2 = t.d == 3 ? (int64_t)K * t.KH : t.KH;
  const int64_t C = P2 * RC;
  const int64_t c0 = (int64_t)local * kDftCB;
  const int cb = (int)std::min<int64_t>(kDftCB, C - c0);
  const T2* tw = reinterpret_cast<const T2*>(f.tw);
  const T* dm = reinterpret_cast<const T*>(ts.der ? f.dmul_der : f.dmul);
  T2* spec = reinterpret_cast<T2*>(f.specA) + c0;
  T2* X = reinterpret_cast<T2*>(dft_smem);
  T2* Y = X + W * kDftCB;
  for (int e = threadIdx.x; e < W * kDftCB; e += blockDim.x) {
    const int cl = e % kDftCB, a = e / kDftCB;
    if (cl < cb) X[e] = spec[(int64_t)a * C + cl];
  }
  __syncthreads();
  // forward along a0 and the multiply: Y[k] = D[k P2 + c / RC] sum_a X[a] w(k, a)
  dft_cplx<T, 2, false>(X, W, kDftCB, cb, K, tw, W, [&](int k, int cl, T2 v) {
    const T dk = dm[(int64_t)k * P2 + (c0 + cl) / RC];
    v.x *= dk;
    v.y *= dk;
    Y[k * kDftCB + cl] = v;
  });
  __syncthreads();
  // inverse along a0: sum_k Y[k] conj(w(k, a))
  dft_cplx<T, 2, true>(Y, K, kDftCB, cb, W, tw, W,
                       [&](int a, int cl, T2 v) { spec[(int64_t)a * C + cl] = v; });
}

// ---------------------------------------------------------------------------
// F3: inverse along the middle axis (d = 3) and the last axis of one plane
// ---------------------------------------------------------------------------
// Shared memory (complex): S2[K][KH][RB], then S1[W][KH][RB] (d = 3); d = 2:
// S2[KH][RB] only.
template <typename T>
__global__ void __launch_bounds__(kDftThreads) k_dft_f3(const DftTasks ts) {
  using T2 = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char dft_smem[];
  int win, local;
  DftTask t;
  if (!dft_task(ts, blockIdx.x, t, win, local)) return;
  const FftWin f = t.tab[win];
  const int RC = ts.RC, RB = t.RB, W = t.W, K = t.K, KH = t.KH;
  const int nrc = RC / RB;
  const int a0 = local / nrc, r0 = (local - a0 * nrc) * RB;
  const T2* tw = reinterpret_cast<const T2*>(f.tw);
  const T2* twh = tw + (int64_t)(KH - 1) * W;
  const T2* spec = reinterpret_cast<const T2*>(f.specA);
  T* grid = reinterpret_cast<T*>(f.grid);
  T2* S2 = reinterpret_cast<T2*>(dft_smem);
  const int P1 = t.d == 3 ? K * KH : KH;              // spectrum values per plane and column
  const T2* src = spec + (int64_t)a0 * P1 * RC + r0;
  for (int e = threadIdx.x; e < P1 * RB; e += blockDim.x) {
    const int rb = e % RB, q = e / RB;
    S2[e] = src[(int64_t)q * RC + rb];
  }
  __syncthreads();
  const int rows = t.d == 3 ? W : 1;
  T* dst = grid + (int64_t)a0 * rows * W * RC + r0;
  if (t.d == 2) {
    // last axis, Hermitian half -> real
    dft_half_real<T, 2>(S2, KH, RB, RB, RB, 0, W, twh, W,
                        [&](int a, int j, T v) { dst[(int64_t)a * RC + j] = v; });
    return;
  }
  // middle axis: S1[a1][k2][rb] = sum_k1 S2[k1][k2][rb] conj(w(k1, a1)); columns j = k2 RB + rb
  T2* S1 = S2 + (int64_t)K * KH * RB;
  dft_cplx<T, 2, true>(S2, K, KH * RB, KH * RB, W, tw, W,
                       [&](int a1, int j, T2 v) { S1[(int64_t)a1 * KH * RB + j] = v; });
  __syncthreads();
  // last axis of every row a1 (columns j = a1 RB + rb)
  dft_half_real<T, 2>(S1, KH, RB, W * RB, RB, KH * RB, W, twh, W, [&](int a2, int j, T v) {
    const int a1 = j / RB, rb = j - a1 * RB;
    dst[((int64_t)a1 * W + a2) * RC + rb] = v;
  });
}

template <typename T>
size_t f1_smem(const DftTask& t) {
  if (t.d == 2) return (size_t)t.W * t.RB * sizeof(T);
  return ((size_t)t.W * t.W * t.RB * sizeof(T) + 15) / 16 * 16 +
         (size_t)t.W * t.KH * t.RB * 2 * sizeof(T);
}
template <typename T>
size_t f3_smem(const DftTask& t) {
  if (t.d == 2) return (size_t)t.KH * t.RB * 2 * sizeof(T);
  return ((size_t)t.K * t.KH + (size_t)t.W * t.KH) * t.RB * 2 * sizeof(T);
}

}  // namespace

bool dft_fused_supported(const FftGroup& g) { return g.d == 2 || g.d == 3; }

template <typename T>
cudaError_t dft_stage(const FftGroup* groups, int n_groups, int der, int RC, cudaStream_t st) {
  if (n_groups < 1 || n_groups > kDftMaxTasks || RC < 1) return cudaErrorInvalidValue;
  DftTasks a{}, b{};
  a.n = b.n = n_groups;
  a.RC = b.RC = RC;
  a.der = b.der = der;
  int ca = 0, cb = 0;
  size_t sm1 = 0, sm2 = 0, sm3 = 0;
  for (int q = 0; q < n_groups; ++q) {
    const FftGroup& g = groups[q];
    if (!dft_fused_supported(g)) return cudaErrorInvalidValue;
    DftTask t{g.tab, g.count, g.d, g.N, g.W, g.N + 1, g.N / 2 + 1, RC, 0, 0};
    if (g.d == 3) {
      // columns per plane: the widest divisor of RC in {8, 4, 2, 1} that fits
      for (int rb : {8, 4, 2, 1}) {
        t.RB = rb;
        if (RC % rb == 0 && f1_smem<T>(t) <= kDftSmemCap && f3_smem<T>(t) <= kDftSmemCap) break;
      }
    }
    if (f1_smem<T>(t) > kDftSmemCap || f3_smem<T>(t) > kDftSmemCap) return cudaErrorInvalidValue;
    t.per_win = g.W * (RC / t.RB);
    t.begin = ca;
    a.t[q] = t;
    ca += t.count * t.per_win;
    sm1 = std::max(sm1, f1_smem<T>(t));
    sm3 = std::max(sm3, f3_smem<T>(t));
    const int64_t C = (g.d == 3 ? (int64_t)t.K * t.KH : t.KH) * RC;
    DftTask u = t;
    u.per_win = (int)((C + kDftCB - 1) / kDftCB);
    u.begin = cb;
    b.t[q] = u;
    cb += u.count * u.per_win;
    sm2 = std::max(sm2, (size_t)(t.W + t.K) * kDftCB * 2 * sizeof(T));
  }
  cudaError_t e = cudaFuncSetAttribute(k_dft_f1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dft_f2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dft_f3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
  if (e != cudaSuccess) return e;
  k_dft_f1<T><<<ca, kDftThreads, sm1, st>>>(a);
  k_dft_f2<T><<<cb, kDftThreads, sm2, st>>>(b);
  k_dft_f3<T><<<ca, kDftThreads, sm3, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t dft_stage<float>(const FftGroup*, int, int, int, cudaStream_t);
template cudaError_t dft_stage<double>(const FftGroup*, int, int, int, cudaStream_t);

}  // namespace agp
