// Pruned d-dimensional DFT between the active box of the oversampled grid and
// the spectrum on I_N (Appendix A step 2 and its adjoint), and the spectral
// multiply by the kernel's deconvolved Fourier coefficients (Sec. 3.1 eq. (3.3)).
//
// The grid is non-zero only on the active box a in [0, W) per dimension
// (grid point l = a + lo), and only the frequencies k in [-N/2, N/2] are kept,
// so each one-dimensional transform is a dense K x W (or W x K) complex
// matrix applied along one axis:
//   forward  X[k] = sum_a g[a] exp(-2 pi i k (a + lo) / n_os)
//   inverse  g[a] = sum_k X[k] exp(+2 pi i k (a + lo) / n_os)
// The last axis is real <-> Hermitian half (k_d in [0, N/2]). A thread owns
// one column of the batched transform and a chunk of its outputs (blockIdx.z:
// KC frequencies of a forward pass, a range of grid positions of an inverse
// pass), so that even the small transforms of a d = 2 window fill the GPU;
// the twiddles are read through the read-only cache (every lane of a warp
// reads the same twiddle). Cost is O(W K) per column, a few percent of the
// spreading / interpolation work at the sizes used here.
//
// Every kernel serves a group of windows with the same (d, N, s) -- the
// windows of one plan, or of every problem of a batch -- in one launch:
// blockIdx.y selects the window's entry in a device table of buffer pointers.
#include <algorithm>

#include "agp_internal.cuh"

namespace agp {
namespace {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

// buffer selector: 0 = grid, 1 = specA, 2 = specB
template <typename P>
__device__ __forceinline__ P* buf(const FftWin& f, int sel) {
  return reinterpret_cast<P*>(sel == 0 ? f.grid : (sel == 1 ? f.specA : f.specB));
}

// Forward along the last axis, real -> half spectrum:
// grid [M][W][RC] real -> specA [M][KH][RC] complex, KH = N/2 + 1.
// tw rows are k + N/2 for k in [-N/2, N/2]; rows N/2 .. N are k = 0 .. N/2.
// Outputs per thread of a forward pass with K outputs per column.
__host__ __device__ constexpr int fwd_chunk(int K) { return K <= 33 ? (K + 2) / 3 : (K + 4) / 5; }

template <typename T, int KH>
__global__ void __launch_bounds__(128)
k_fwd_last(const FftWin* __restrict__ tab, int W, int RC, int64_t M) {
  using T2 = typename C2<T>::t;
  constexpr int KC = fwd_chunk(KH);
  const FftWin f = tab[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * RC) return;
  const int64_t m = e / RC;
  const int r = (int)(e - m * RC);
  const int k0 = blockIdx.z * KC;                  // this thread's frequencies k0 .. k0 + KC - 1
  const T2* twh = reinterpret_cast<const T2*>(f.tw) + (int64_t)(KH - 1) * W;   // row of k = 0
  T re[KC], im[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) re[k] = im[k] = T(0);
  const T* src = buf<const T>(f, 0) + m * W * RC + r;
  for (int a = 0; a < W; ++a) {
    const T x = src[(int64_t)a * RC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const T2 t = __ldg(twh + (int64_t)min(k0 + k, KH - 1) * W + a);
      re[k] = fma(x, t.x, re[k]);
      im[k] = fma(x, t.y, im[k]);
    }
  }
  T2* dst = buf<T2>(f, 1) + m * KH * RC + r;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    if (k0 + k >= KH) break;
    T2 v;
    v.x = re[k];
    v.y = im[k];
    dst[(int64_t)(k0 + k) * RC] = v;
  }
}

// Forward along a non-last axis, complex -> complex: [M][W][I] -> [M][K][I], K = N + 1.
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_fwd_mid(const FftWin* __restrict__ tab, int src_sel, int dst_sel, int W, int64_t M, int64_t I) {
  using T2 = typename C2<T>::t;
  const FftWin f = tab[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * I) return;
  constexpr int KC = fwd_chunk(K);
  const int64_t m = e / I;
  const int64_t i = e - m * I;
  const int k0 = blockIdx.z * KC;
  const T2* tw = reinterpret_cast<const T2*>(f.tw);
  T re[KC], im[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) re[k] = im[k] = T(0);
  const T2* src = buf<const T2>(f, src_sel) + m * W * I + i;
  for (int a = 0; a < W; ++a) {
    const T2 x = src[(int64_t)a * I];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const T2 t = __ldg(tw + (int64_t)min(k0 + k, K - 1) * W + a);
      re[k] = fma(x.x, t.x, re[k]);
      re[k] = fma(-x.y, t.y, re[k]);
      im[k] = fma(x.x, t.y, im[k]);
      im[k] = fma(x.y, t.x, im[k]);
    }
  }
  T2* dst = buf<T2>(f, dst_sel) + m * K * I + i;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    if (k0 + k >= K) break;
    T2 v;
    v.x = re[k];
    v.y = im[k];
    dst[(int64_t)(k0 + k) * I] = v;
  }
}

// Inverse along a non-last axis: [M][K][I] -> [M][W][I] (conjugate twiddles).
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_inv_mid(const FftWin* __restrict__ tab, int src_sel, int dst_sel, int W, int64_t M, int64_t I) {
  using T2 = typename C2<T>::t;
  const FftWin f = tab[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * I) return;
  const int64_t m = e / I;
  const int64_t i = e - m * I;
  const T2* tw = reinterpret_cast<const T2*>(f.tw);
  T xr[K], xi[K];
  const T2* src = buf<const T2>(f, src_sel) + m * K * I + i;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T2 x = src[(int64_t)k * I];
    xr[k] = x.x;
    xi[k] = x.y;
  }
  T2* dst = buf<T2>(f, dst_sel) + m * W * I + i;
  const int aw = (W + gridDim.z - 1) / gridDim.z, a1 = min(W, (int)(blockIdx.z + 1) * aw);
  for (int a = blockIdx.z * aw; a < a1; ++a) {
    T re = T(0), im = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T2 t = __ldg(tw + (int64_t)k * W + a);   // conj(t) = (t.x, -t.y)
      re = fma(xr[k], t.x, re);
      re = fma(xi[k], t.y, re);
      im = fma(xi[k], t.x, im);
      im = fma(-xr[k], t.y, im);
    }
    T2 v;
    v.x = re;
    v.y = im;
    dst[(int64_t)a * I] = v;
  }
}

// Inverse along the last axis, Hermitian half -> real grid:
// g[a] = Re X_0 + 2 sum_{k=1}^{N/2} Re(X_k exp(+2 pi i k (a + lo) / n_os)).
template <typename T, int KH>
__global__ void __launch_bounds__(128)
k_inv_last(const FftWin* __restrict__ tab, int src_sel, int W, int RC, int64_t M) {
  using T2 = typename C2<T>::t;
  const FftWin f = tab[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * RC) return;
  const int64_t m = e / RC;
  const int r = (int)(e - m * RC);
  const T2* twh = reinterpret_cast<const T2*>(f.tw) + (int64_t)(KH - 1) * W;
  T xr[KH], xi[KH];
  const T2* src = buf<const T2>(f, src_sel) + m * KH * RC + r;
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    const T2 x = src[(int64_t)k * RC];
    const T s = (k == 0) ? T(1) : T(2);
    xr[k] = s * x.x;
    xi[k] = s * x.y;
  }
  T* dst = buf<T>(f, 0) + m * W * RC + r;
  const int aw = (W + gridDim.z - 1) / gridDim.z, a1 = min(W, (int)(blockIdx.z + 1) * aw);
  for (int a = blockIdx.z * aw; a < a1; ++a) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      const T2 t = __ldg(twh + (int64_t)k * W + a);
      acc = fma(xr[k], t.x, acc);
      acc = fma(xi[k], t.y, acc);
    }
    dst[(int64_t)a * RC] = acc;
  }
}

template <typename T>
__global__ void k_spec_mul(const FftWin* __restrict__ tab, int sel, int der, int RC, int64_t total) {
  using T2 = typename C2<T>::t;
  const FftWin f = tab[blockIdx.y];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const T d = reinterpret_cast<const T*>(der ? f.dmul_der : f.dmul)[e / RC];
  T2* spec = buf<T2>(f, sel);
  T2 v = spec[e];
  v.x *= d;
  v.y *= d;
  spec[e] = v;
}

// zero the grids of every window of a group: [grid_elems * RC] each
template <typename T>
__global__ void k_zero_grids(const FftWin* __restrict__ tab, int64_t total) {
  const FftWin f = tab[blockIdx.y];
  T* g = reinterpret_cast<T*>(f.grid);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    g[e] = T(0);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

inline int64_t powi(int64_t b, int e) {
  int64_t r = 1;
  for (int t = 0; t < e; ++t) r *= b;
  return r;
}

// Grid-position chunks of an inverse pass with `columns` columns in all: about
// 128k threads in flight, chunks of at least 8 positions.
unsigned inv_chunks(int64_t columns, int W) {
  int64_t z = (131072 + columns - 1) / columns;
  z = std::min<int64_t>(z, std::max(1, W / 8));
  return (unsigned)std::max<int64_t>(z, 1);
}

template <typename T, int N>
cudaError_t forward_n(const FftGroup& g, int RC, cudaStream_t st) {
  constexpr int K = N + 1, KH = N / 2 + 1;
  const int W = g.W;
  const int64_t M = powi(W, g.d - 1);
  k_fwd_last<T, KH><<<dim3(blocks_for(M * RC, 128), g.count, (KH + fwd_chunk(KH) - 1) / fwd_chunk(KH)),
                      128, 0, st>>>(g.tab, W, RC, M);
  // remaining axes from the second-to-last down to the first (ping-pong A/B)
  int src = 1, dst = 2;
  int64_t I = (int64_t)KH * RC;
  for (int axis = g.d - 2; axis >= 0; --axis) {
    const int64_t Mo = powi(W, axis);
    k_fwd_mid<T, K><<<dim3(blocks_for(Mo * I, 128), g.count, (K + fwd_chunk(K) - 1) / fwd_chunk(K)),
                      128, 0, st>>>(g.tab, src, dst, W, Mo, I);
    I *= K;
    const int t = src;
    src = dst;
    dst = t;
  }
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t inverse_n(const FftGroup& g, int RC, cudaStream_t st) {
  constexpr int K = N + 1, KH = N / 2 + 1;
  const int W = g.W;
  // The forward pass leaves the spectrum in A for odd d and in B for even d.
  int src = (g.d % 2) ? 1 : 2, dst = (g.d % 2) ? 2 : 1;
  int64_t I = (int64_t)KH * RC * powi(K, g.d - 1);
  for (int axis = 0; axis <= g.d - 2; ++axis) {
    I /= K;
    const int64_t Mo = powi(W, axis);
    k_inv_mid<T, K><<<dim3(blocks_for(Mo * I, 128), g.count, inv_chunks(Mo * I * g.count, W)), 128,
                      0, st>>>(g.tab, src, dst, W, Mo, I);
    const int t = src;
    src = dst;
    dst = t;
  }
  const int64_t M = powi(W, g.d - 1);
  k_inv_last<T, KH><<<dim3(blocks_for(M * RC, 128), g.count, inv_chunks(M * RC * g.count, W)), 128,
                       0, st>>>(g.tab, src, W, RC, M);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t fft_forward(const FftGroup& g, int RC, cudaStream_t st) {
  switch (g.N) {
    case 8: return forward_n<T, 8>(g, RC, st);
    case 16: return forward_n<T, 16>(g, RC, st);
    case 32: return forward_n<T, 32>(g, RC, st);
    case 64: return forward_n<T, 64>(g, RC, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t fft_inverse(const FftGroup& g, int RC, cudaStream_t st) {
  switch (g.N) {
    case 8: return inverse_n<T, 8>(g, RC, st);
    case 16: return inverse_n<T, 16>(g, RC, st);
    case 32: return inverse_n<T, 32>(g, RC, st);
    case 64: return inverse_n<T, 64>(g, RC, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t spectral_multiply(const FftGroup& g, int der, int RC, cudaStream_t st) {
  const int64_t total = g.dmul_elems * RC;
  k_spec_mul<T><<<dim3(blocks_for(total, 256), g.count), 256, 0, st>>>(g.tab, (g.d % 2) ? 1 : 2,
                                                                       der, RC, total);
  return cudaGetLastError();
}

template <typename T>
cudaError_t zero_grids(const FftGroup& g, int RC, cudaStream_t st) {
  const int64_t total = g.grid_elems * RC;
  const unsigned bx = (unsigned)std::min<int64_t>(blocks_for(total, 256), 1024);
  k_zero_grids<T><<<dim3(bx, g.count), 256, 0, st>>>(g.tab, total);
  return cudaGetLastError();
}

template cudaError_t fft_forward<float>(const FftGroup&, int, cudaStream_t);
template cudaError_t fft_forward<double>(const FftGroup&, int, cudaStream_t);
template cudaError_t fft_inverse<float>(const FftGroup&, int, cudaStream_t);
template cudaError_t fft_inverse<double>(const FftGroup&, int, cudaStream_t);
template cudaError_t spectral_multiply<float>(const FftGroup&, int, int, cudaStream_t);
template cudaError_t spectral_multiply<double>(const FftGroup&, int, int, cudaStream_t);
template cudaError_t zero_grids<float>(const FftGroup&, int, cudaStream_t);
template cudaError_t zero_grids<double>(const FftGroup&, int, cudaStream_t);

}  // namespace agp
