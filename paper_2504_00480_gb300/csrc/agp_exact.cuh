// Exact-kernel helpers shared by the landmark (Nystrom) and AFN
// preconditioners: caller-order coordinates, farthest point sampling, the
// exact additive kernel (Sec. 2.1) in FP64, and small dense FP64
// factorisations on one CTA. Kernels live in an anonymous namespace, so every
// translation unit that includes this header gets its own copies.
#pragma once

#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

#define AGP_CUDA(call)                                             \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);          \
  } while (0)
#define AGP_TRY(call)                                              \
  do {                                                             \
    agp_status s_ = (call);                                        \
    if (s_ != AGP_OK) return s_;                                   \
  } while (0)

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// sorted [d][n] coordinates -> caller order [d][n]
template <typename T>
__global__ void k_unsort(const T* __restrict__ xs, const int32_t* __restrict__ perm, int64_t n,
                         int d, T* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * d) return;
  const int t = (int)(e / n);
  const int64_t q = e - (int64_t)t * n;
  out[(int64_t)t * n + perm[q]] = xs[e];
}

__global__ void k_fill_double(double* __restrict__ p, int64_t n, double v) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) p[e] = v;
}

// Farthest point sampling (Sec. 2.3), one step in two launches. k_fps_dist
// folds landmark chosen[step - 1] into the running minimum squared distances
// and writes each block's farthest point; k_fps_pick reduces the blocks'
// candidates into chosen[step]. Distances and the comparison are FP64: the
// squared distance is the plainly rounded sum ((u_0^2 + u_1^2) + u_2^2) of
// the coordinate differences (no fused multiply-add, so the choice does not
// depend on how the compiler contracts it); the farthest point is the one
// with the largest distance, the lowest index among equal distances.
__device__ __forceinline__ void fps_better(double& bd, int64_t& bi, double od, int64_t oi) {
  if (od > bd || (od == bd && oi < bi)) {
    bd = od;
    bi = oi;
  }
}

constexpr int kFpsThreads = 256;

// block-wide (distance, index) maximum of the calling block, valid in thread 0
__device__ void fps_block_best(double& bd, int64_t& bi) {
  __shared__ double sd[kFpsThreads / 32];
  __shared__ int64_t si[kFpsThreads / 32];
  for (int o = 16; o > 0; o >>= 1)
    fps_better(bd, bi, __shfl_xor_sync(0xFFFFFFFFu, bd, o), __shfl_xor_sync(0xFFFFFFFFu, bi, o));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    sd[warp] = bd;
    si[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < kFpsThreads / 32; ++w) fps_better(bd, bi, sd[w], si[w]);
}

template <typename T>
__global__ void __launch_bounds__(kFpsThreads)
k_fps_dist(const T* __restrict__ x, int64_t n, int d, const int32_t* __restrict__ chosen, int step,
           double* __restrict__ dist, double* __restrict__ cand_d, int64_t* __restrict__ cand_i) {
  const int64_t last = chosen[step - 1];
  double xl[3] = {0, 0, 0};
  for (int t = 0; t < d; ++t) xl[t] = (double)x[(int64_t)t * n + last];
  double bd = -1.0;
  int64_t bi = n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d2 = 0.0;
    for (int t = 0; t < d; ++t) {
      const double u = (double)x[(int64_t)t * n + i] - xl[t];
      d2 = __dadd_rn(d2, __dmul_rn(u, u));
    }
    const double m = fmin(dist[i], d2);
    dist[i] = m;
    fps_better(bd, bi, m, i);
  }
  fps_block_best(bd, bi);
  if (threadIdx.x == 0) {
    cand_d[blockIdx.x] = bd;
    cand_i[blockIdx.x] = bi;
  }
}

__global__ void __launch_bounds__(kFpsThreads)
k_fps_pick(const double* __restrict__ cand_d, const int64_t* __restrict__ cand_i, int nb,
           int32_t* __restrict__ chosen, int step) {
  double bd = -1.0;
  int64_t bi = INT64_MAX;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) fps_better(bd, bi, cand_d[b], cand_i[b]);
  fps_block_best(bd, bi);
  if (threadIdx.x == 0) chosen[step] = (int32_t)bi;
}

// B[i][j] = sigma_f^2 sum_s kappa_s(|x_i^s - x_{L_j}^s|) (exact kernel, Sec. 2.1)
template <typename T>
struct WinPts {
  const T* x;   // caller order [d][n]
  int d;
};

// sum_s kappa_s(|x_i^s - x_l^s|) (der = 0) or its ell-derivative (der = 1;
// Sec. 2.1 eq. (2.3) and kernel_value), exact kernel in FP64 from the
// plan-precision coordinates
template <typename T>
__device__ double kernel_sum(const WinPts<T>* __restrict__ wp, int P, int64_t n, int64_t i,
                             int64_t l, int kernel, double ell, int der) {
  double s = 0.0;
  for (int w = 0; w < P; ++w) {
    const WinPts<T> p = wp[w];
    double r2 = 0.0;
    for (int t = 0; t < p.d; ++t) {
      const double u = (double)p.x[(int64_t)t * n + i] - (double)p.x[(int64_t)t * n + l];
      r2 += u * u;
    }
    s += kernel_value(kernel, r2, ell, der);
  }
  return s;
}

// B[i][j] = sigma_f^2 kernel_sum(i, L_j) (or its ell-derivative), [n][k]
template <typename T>
__global__ void k_kernel_cols(const WinPts<T>* __restrict__ wp, int P, int64_t n,
                              const int32_t* __restrict__ lm, int k, int kernel, double ell,
                              double sf2, int der, T* __restrict__ B) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t i = e / k;
  const int j = (int)(e - i * k);
  B[e] = (T)(sf2 * kernel_sum<T>(wp, P, n, i, lm[j], kernel, ell, der));
}

// K_LL[a][b] = sigma_f^2 kernel_sum(L_a, L_b) + delta [a == b] in FP64 (or the
// ell-derivative block with delta = 0)
template <typename T>
__global__ void k_kernel_block(const WinPts<T>* __restrict__ wp, int P, int64_t n,
                               const int32_t* __restrict__ lm, int k, int kernel, double ell,
                               double sf2, int der, double delta, double* __restrict__ K) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int a = e / k, b = e - a * k;
  K[e] = sf2 * kernel_sum<T>(wp, P, n, lm[a], lm[b], kernel, ell, der) + (a == b ? delta : 0.0);
}

// A[j][j] += delta
__global__ void k_shift_diag(double* __restrict__ A, int k, double delta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) A[(int64_t)j * k + j] += delta;
}

__global__ void k_diag(const double* __restrict__ A, int k, double* __restrict__ d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) d[j] = A[(int64_t)j * k + j];
}

// In-place lower Cholesky factor of G (k x k, FP64) by one CTA; flag = 1 on a
// non-positive pivot.
__global__ void __launch_bounds__(1024) k_cholesky(double* __restrict__ G, int k, int* flag) {
  for (int j = 0; j < k; ++j) {
    __syncthreads();
    const double piv = G[(int64_t)j * k + j];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) *flag = 1;
      return;
    }
    const double lj = sqrt(piv);
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) G[(int64_t)i * k + j] /= lj;
    if (threadIdx.x == 0) G[(int64_t)j * k + j] = lj;
    __syncthreads();
    const int m = k - j - 1;   // trailing lower triangle, rows/cols j+1 .. k-1
    for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
      const int ii = j + 1 + (int)(e / m), ll = j + 1 + (int)(e % m);
      if (ll <= ii) G[(int64_t)ii * k + ll] -= G[(int64_t)ii * k + j] * G[(int64_t)ll * k + j];
    }
  }
}

// Column j of L^{-1} by forward substitution (thread per column).
__global__ void k_tri_inverse(const double* __restrict__ L, int k, double* __restrict__ Li) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  for (int i = 0; i < j; ++i) Li[(int64_t)i * k + j] = 0.0;
  for (int i = j; i < k; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int m = j; m < i; ++m) s -= L[(int64_t)i * k + m] * Li[(int64_t)m * k + j];
    Li[(int64_t)i * k + j] = s / L[(int64_t)i * k + i];
  }
}

// Ginv = L^{-T} L^{-1}
__global__ void k_gram_inverse(const double* __restrict__ Li, int k, double* __restrict__ Gi) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int a = e / k, b = e - a * k;
  double s = 0.0;
  for (int m = max(a, b); m < k; ++m) s += Li[(int64_t)m * k + a] * Li[(int64_t)m * k + b];
  Gi[e] = s;
}

}  // namespace

// Caller-order coordinates of every window (freed with the object).
template <typename T>
struct CallerPoints {
  std::vector<T*> xo;
  std::vector<WinPts<T>> wp;
  cudaStream_t st = nullptr;
  ~CallerPoints() {
    for (T* p : xo)
      if (p) cudaFreeAsync(p, st);
  }
};

// Caller-order [d][n] coordinates of every window, in the plan precision.
template <typename T>
agp_status caller_points(agp_plan_s* pl, CallerPoints<T>& cp, cudaStream_t st);
// Landmarks: ceil(k_req / P) per window by farthest point sampling, merged
// into a sorted set without repeats (host vector).
template <typename T>
agp_status select_landmarks(agp_plan_s* pl, const CallerPoints<T>& cp, int k_req,
                            std::vector<int32_t>& all, cudaStream_t st);

}  // namespace agp
