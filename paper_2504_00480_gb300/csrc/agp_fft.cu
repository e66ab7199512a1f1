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
// The last axis is real <-> Hermitian half (k_d in [0, N/2]). Each thread owns
// one column of the batched transform and keeps its K outputs in registers;
// the twiddles are read through the read-only cache (every lane of a warp
// reads the same twiddle). Cost is O(W K) per column, a few percent of the
// spreading / interpolation work at the sizes used here.
#include "agp_internal.cuh"

namespace agp {
namespace {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

// Forward along the last axis, real -> half spectrum:
// in [M][W][RC] real, out [M][KH][RC] complex, KH = N/2 + 1.
// tw rows are k + N/2 for k in [-N/2, N/2]; rows N/2 .. N are k = 0 .. N/2.
template <typename T, int KH>
__global__ void __launch_bounds__(128)
k_fwd_last(const T* __restrict__ in, typename C2<T>::t* __restrict__ out,
           const typename C2<T>::t* __restrict__ tw, int W, int RC, int64_t M) {
  using T2 = typename C2<T>::t;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * RC) return;
  const int64_t m = e / RC;
  const int r = (int)(e - m * RC);
  const T2* twh = tw + (int64_t)(KH - 1) * W;   // row of k = 0
  T re[KH], im[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) re[k] = im[k] = T(0);
  const T* src = in + m * W * RC + r;
  for (int a = 0; a < W; ++a) {
    const T x = src[(int64_t)a * RC];
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      const T2 t = __ldg(twh + (int64_t)k * W + a);
      re[k] = fma(x, t.x, re[k]);
      im[k] = fma(x, t.y, im[k]);
    }
  }
  T2* dst = out + m * KH * RC + r;
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    T2 v;
    v.x = re[k];
    v.y = im[k];
    dst[(int64_t)k * RC] = v;
  }
}

// Forward along a non-last axis, complex -> complex:
// in [M][W][I], out [M][K][I], K = N + 1.
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_fwd_mid(const typename C2<T>::t* __restrict__ in, typename C2<T>::t* __restrict__ out,
          const typename C2<T>::t* __restrict__ tw, int W, int64_t M, int64_t I) {
  using T2 = typename C2<T>::t;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * I) return;
  const int64_t m = e / I;
  const int64_t i = e - m * I;
  T re[K], im[K];
#pragma unroll
  for (int k = 0; k < K; ++k) re[k] = im[k] = T(0);
  const T2* src = in + m * W * I + i;
  for (int a = 0; a < W; ++a) {
    const T2 x = src[(int64_t)a * I];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T2 t = __ldg(tw + (int64_t)k * W + a);
      re[k] = fma(x.x, t.x, re[k]);
      re[k] = fma(-x.y, t.y, re[k]);
      im[k] = fma(x.x, t.y, im[k]);
      im[k] = fma(x.y, t.x, im[k]);
    }
  }
  T2* dst = out + m * K * I + i;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T2 v;
    v.x = re[k];
    v.y = im[k];
    dst[(int64_t)k * I] = v;
  }
}

// Inverse along a non-last axis: in [M][K][I] -> out [M][W][I] (conjugate twiddles).
template <typename T, int K>
__global__ void __launch_bounds__(128)
k_inv_mid(const typename C2<T>::t* __restrict__ in, typename C2<T>::t* __restrict__ out,
          const typename C2<T>::t* __restrict__ tw, int W, int64_t M, int64_t I) {
  using T2 = typename C2<T>::t;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * I) return;
  const int64_t m = e / I;
  const int64_t i = e - m * I;
  T xr[K], xi[K];
  const T2* src = in + m * K * I + i;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T2 x = src[(int64_t)k * I];
    xr[k] = x.x;
    xi[k] = x.y;
  }
  T2* dst = out + m * W * I + i;
  for (int a = 0; a < W; ++a) {
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

// Inverse along the last axis, Hermitian half -> real:
// g[a] = Re X_0 + 2 sum_{k=1}^{N/2} Re(X_k exp(+2 pi i k (a + lo) / n_os)).
template <typename T, int KH>
__global__ void __launch_bounds__(128)
k_inv_last(const typename C2<T>::t* __restrict__ in, T* __restrict__ out,
           const typename C2<T>::t* __restrict__ tw, int W, int RC, int64_t M) {
  using T2 = typename C2<T>::t;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M * RC) return;
  const int64_t m = e / RC;
  const int r = (int)(e - m * RC);
  const T2* twh = tw + (int64_t)(KH - 1) * W;
  T xr[KH], xi[KH];
  const T2* src = in + m * KH * RC + r;
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    const T2 x = src[(int64_t)k * RC];
    const T f = (k == 0) ? T(1) : T(2);
    xr[k] = f * x.x;
    xi[k] = f * x.y;
  }
  T* dst = out + m * W * RC + r;
  for (int a = 0; a < W; ++a) {
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
__global__ void k_spec_mul(typename C2<T>::t* __restrict__ spec, const T* __restrict__ dmul,
                           int RC, int64_t total) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const T d = dmul[e / RC];
  typename C2<T>::t v = spec[e];
  v.x *= d;
  v.y *= d;
  spec[e] = v;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T, int N>
cudaError_t forward_n(const Window& w, int RC, cudaStream_t st) {
  using T2 = typename C2<T>::t;
  constexpr int K = N + 1, KH = N / 2 + 1;
  const int W = w.W;
  const T2* tw = reinterpret_cast<const T2*>(w.tw);
  const T* g = reinterpret_cast<const T*>(w.grid);
  T2* A = reinterpret_cast<T2*>(w.specA);
  T2* B = reinterpret_cast<T2*>(w.specB);
  int64_t M = 1;
  for (int t = 0; t < w.d - 1; ++t) M *= W;
  k_fwd_last<T, KH><<<blocks_for(M * RC, 128), 128, 0, st>>>(g, A, tw, W, RC, M);
  // remaining axes from the second-to-last down to the first
  T2* src = A;
  T2* dst = B;
  int64_t I = (int64_t)KH * RC;
  for (int axis = w.d - 2; axis >= 0; --axis) {
    int64_t Mo = 1;
    for (int t = 0; t < axis; ++t) Mo *= W;
    k_fwd_mid<T, K><<<blocks_for(Mo * I, 128), 128, 0, st>>>(src, dst, tw, W, Mo, I);
    I *= K;
    T2* tmp = src;
    src = dst;
    dst = tmp;
  }
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t inverse_n(const Window& w, int RC, cudaStream_t st) {
  using T2 = typename C2<T>::t;
  constexpr int K = N + 1, KH = N / 2 + 1;
  const int W = w.W;
  const T2* tw = reinterpret_cast<const T2*>(w.tw);
  T* g = reinterpret_cast<T*>(w.grid);
  T2* A = reinterpret_cast<T2*>(w.specA);
  T2* B = reinterpret_cast<T2*>(w.specB);
  // The forward pass leaves the spectrum in A for odd d and in B for even d.
  T2* src = (w.d % 2) ? A : B;
  T2* dst = (w.d % 2) ? B : A;
  int64_t I = (int64_t)KH * RC;
  for (int t = 0; t < w.d - 1; ++t) I *= K;
  for (int axis = 0; axis <= w.d - 2; ++axis) {
    I /= K;
    int64_t Mo = 1;
    for (int t = 0; t < axis; ++t) Mo *= W;
    k_inv_mid<T, K><<<blocks_for(Mo * I, 128), 128, 0, st>>>(src, dst, tw, W, Mo, I);
    T2* tmp = src;
    src = dst;
    dst = tmp;
  }
  int64_t M = 1;
  for (int t = 0; t < w.d - 1; ++t) M *= W;
  k_inv_last<T, KH><<<blocks_for(M * RC, 128), 128, 0, st>>>(src, g, tw, W, RC, M);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t fft_forward(const Window& w, int RC, cudaStream_t st) {
  switch (w.N) {
    case 8: return forward_n<T, 8>(w, RC, st);
    case 16: return forward_n<T, 16>(w, RC, st);
    case 32: return forward_n<T, 32>(w, RC, st);
    case 64: return forward_n<T, 64>(w, RC, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t fft_inverse(const Window& w, int RC, cudaStream_t st) {
  switch (w.N) {
    case 8: return inverse_n<T, 8>(w, RC, st);
    case 16: return inverse_n<T, 16>(w, RC, st);
    case 32: return inverse_n<T, 32>(w, RC, st);
    case 64: return inverse_n<T, 64>(w, RC, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t spectral_multiply(const Window& w, const void* dmul, int RC, cudaStream_t st) {
  using T2 = typename C2<T>::t;
  T2* spec = reinterpret_cast<T2*>((w.d % 2) ? w.specA : w.specB);
  const int64_t total = w.dmul_elems * RC;
  k_spec_mul<T><<<blocks_for(total, 256), 256, 0, st>>>(spec, reinterpret_cast<const T*>(dmul),
                                                        RC, total);
  return cudaGetLastError();
}

template cudaError_t fft_forward<float>(const Window&, int, cudaStream_t);
template cudaError_t fft_forward<double>(const Window&, int, cudaStream_t);
template cudaError_t fft_inverse<float>(const Window&, int, cudaStream_t);
template cudaError_t fft_inverse<double>(const Window&, int, cudaStream_t);
template cudaError_t spectral_multiply<float>(const Window&, const void*, int, cudaStream_t);
template cudaError_t spectral_multiply<double>(const Window&, const void*, int, cudaStream_t);

}  // namespace agp
