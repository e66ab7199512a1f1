// Landmark (Nystrom) preconditioner for batched PCG -- the (1,1)-block part of
// the paper's additive AFN preconditioner (Sec. 2.3): landmarks are chosen by
// farthest point sampling (FPS) in every feature window and merged; with
// B = K_{:,L} (the kernel part sigma_f^2 sum_s K_s, exact kernel) and K_LL
// its landmark rows, evaluated in FP64, plus delta I (a safeguard when the
// landmarks outnumber the kernel's numerical rank, see precond_build),
//     M = B K_LL^{-1} B^T + sigma_eps^2 I,
//     M^{-1} = sigma_eps^{-2} (I - B G^{-1} B^T),  G = sigma_eps^2 K_LL + B^T B
// (Woodbury identity). G is k x k (k <= 512) and inverted once in FP64 by a
// Cholesky factorisation; applying M^{-1} to an [n][R] block costs two skinny
// products with B.
//
// Accuracy: M^{-1} r = sigma_eps^{-2} (r - B t2) cancels heavily where r lies
// in the landmark space, so relative errors of B t2 are amplified by up to
// kappa(M) ~ |K| / sigma_eps^2; with plain FP32 sums the preconditioned CG
// stalls. FP32 plans therefore split the FP64 inputs into hi + lo FP32 parts
// and accumulate every product with B, and the Gram matrix B^T B, with the
// compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm Dot2): about twice
// the FP32 precision at ~10 FP32 operations per term, instead of FP64
// arithmetic, which runs at a small fraction of the FP32 rate on this part.
//
// FPS: the first landmark of a window is the caller's point 0; each next one
// maximises the distance to the landmarks chosen so far (ties: lowest index),
// found with a packed (distance, index) atomic maximum.
#include <algorithm>
#include <cmath>
#include <vector>

#include "agp_exact.cuh"

namespace agp {
namespace {

// One step of Dot2: (s, c) += a * b with the product split exactly into
// p + e and an error-free two-sum of s and p; the rounding errors collect in
// c. The value is s + c. The _rn intrinsics are never fused or reordered.
__device__ __forceinline__ void dot2_add(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  c = __fadd_rn(c, __fadd_rn(q, e));
  s = t;
}

// x (FP64) -> hi = fl32(x), lo = fl32(x - hi)
__global__ void k_split(const double* __restrict__ x, int64_t m, float* __restrict__ hi,
                        float* __restrict__ lo) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m) return;
  const double v = x[e];
  const float h = __double2float_rn(v);
  hi[e] = h;
  lo[e] = __double2float_rn(v - (double)h);
}

// G += B^T C over a slice of rows (C = B for the Gram matrix): 32 x 32 output
// tile per CTA (blockIdx.x, y),
// row slices over blockIdx.z, added to G with FP64 atomics. FP64 plans: FP64
// FMAs; FP32 plans: Dot2 over the whole slice (the products of FP32 entries
// are split exactly).
template <typename T>
__global__ void __launch_bounds__(1024)
k_gram(const T* __restrict__ B, const T* __restrict__ C, int64_t n, int k, int64_t rows_per_slice,
       double* __restrict__ G) {
  __shared__ T sa[64][33];
  __shared__ T sb[64][33];
  const int ta = threadIdx.x / 32, tb = threadIdx.x % 32;
  const int a = blockIdx.x * 32 + ta, b = blockIdx.y * 32 + tb;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_slice;
  const int64_t r1 = min(n, r0 + rows_per_slice);
  double acc = 0.0;
  float s = 0.0f, c = 0.0f;
  for (int64_t rb = r0; rb < r1; rb += 64) {
    for (int e = threadIdx.x; e < 64 * 32; e += 1024) {
      const int rr = e / 32, cc = e % 32;
      const int64_t row = rb + rr;
      const int ca = blockIdx.x * 32 + cc, cb = blockIdx.y * 32 + cc;
      sa[rr][cc] = (row < r1 && ca < k) ? B[row * k + ca] : T(0);
      sb[rr][cc] = (row < r1 && cb < k) ? C[row * k + cb] : T(0);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
#pragma unroll 8
      for (int rr = 0; rr < 64; ++rr) dot2_add(s, c, sa[rr][ta], sb[rr][tb]);
    } else {
#pragma unroll 8
      for (int rr = 0; rr < 64; ++rr) acc = fma((double)sa[rr][ta], (double)sb[rr][tb], acc);
    }
    __syncthreads();
  }
  if constexpr (sizeof(T) == 4) acc = (double)s + (double)c;
  if (a < k && b < k) atomicAdd(G + (int64_t)a * k + b, acc);
}

// out = s a + b (m values)
__global__ void k_axpy(const double* __restrict__ a, double s, const double* __restrict__ b,
                       int64_t m, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) out[e] = s * a[e] + b[e];
}

// Apply step 1: partial[z][j][r] = sum over row slice z of B[i][j] * X[i][r].
// CTA: 32 landmark columns (4 per warp) x 32 right-hand sides (lanes), so each
// block of X rows is read once per 32 landmarks. FP64 plans: FP64 FMAs; FP32
// plans: Dot2 on X's hi part plus plain FMAs on its lo part.
template <typename T>
__global__ void __launch_bounds__(256)
k_pc_bt(const T* __restrict__ B, const double* __restrict__ X, const float* __restrict__ Xh,
        const float* __restrict__ Xl, int64_t n, int k, int R, int64_t rows_per_slice,
        double* __restrict__ partial) {
  const int r = threadIdx.x % 32;
  const int j0 = blockIdx.x * 32 + (threadIdx.x / 32) * 4;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t r1 = min(n, r0 + rows_per_slice);
  if (r >= R) return;
  int nq = k - j0;
  nq = nq < 0 ? 0 : (nq > 4 ? 4 : nq);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if constexpr (sizeof(T) == 4) {
    float s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
    for (int64_t i = r0; i < r1; ++i) {
      const float xh = Xh[i * R + r], xl = Xl[i * R + r];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nq) {
          const float b = __ldg(B + i * k + j0 + q);
          dot2_add(s[q], c[q], b, xh);
          sl[q] = __fmaf_rn(b, xl, sl[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = (double)s[q] + (double)c[q] + (double)sl[q];
  } else {
    for (int64_t i = r0; i < r1; ++i) {
      const double x = X[i * R + r];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nq) acc[q] = fma((double)__ldg(B + i * k + j0 + q), x, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < nq) partial[((int64_t)blockIdx.y * k + j0 + q) * R + r] = acc[q];
}

// Apply step 2 (two launches): phase 0 sums the slices, t1 = sum_z partial[z];
// phase 1 multiplies, t2 = Ginv t1 (k x R, FP64), stored as FP64 (FP64 plans)
// or as hi and lo FP32 parts (FP32 plans).
template <typename T>
__global__ void k_pc_mid(const double* __restrict__ partial, int nz, const double* __restrict__ Gi,
                         int k, int R, int phase, double* __restrict__ t1, void* __restrict__ t2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * R) return;
  if (phase == 0) {   // reduce the slices
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += partial[(int64_t)z * k * R + e];
    t1[e] = s;
  } else {            // multiply by Ginv
    const int a = e / R, r = e - a * R;
    double s = 0.0;
    for (int b = 0; b < k; ++b) s += Gi[(int64_t)a * k + b] * t1[(int64_t)b * R + r];
    if constexpr (sizeof(T) == 4) {
      float* t2f = static_cast<float*>(t2);
      const float h = __double2float_rn(s);
      t2f[e] = h;
      t2f[(int64_t)k * R + e] = __double2float_rn(s - (double)h);
    } else {
      static_cast<double*>(t2)[e] = s;
    }
  }
}

// Apply step 3: Y[i][r] = inv_s2 (X[i][r] - sum_j B[i][j] t2[j][r]); a warp per
// row, lanes = right-hand sides, t2 staged in shared memory. FP32 plans: Dot2
// on t2's hi part plus FMAs on its lo part, the subtraction in FP64.
template <typename T>
__global__ void __launch_bounds__(256)
k_pc_out(const T* __restrict__ B, const double* __restrict__ X, const void* __restrict__ t2,
         int64_t n, int k, int R, double inv_s2, double* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NP = sizeof(T) == 4 ? 2 : 1;   // hi, lo parts (FP32) or the FP64 values
  T* st2 = reinterpret_cast<T*>(smem_raw);     // [NP][k][R]
  for (int e = threadIdx.x; e < NP * k * R; e += blockDim.x) st2[e] = static_cast<const T*>(t2)[e];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  if (lane >= R) return;
  for (int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; i < n; i += (int64_t)gridDim.x * 8) {
    const T* brow = B + i * k;
    double bt;
    if constexpr (sizeof(T) == 4) {
      float s = 0.0f, c = 0.0f, sl = 0.0f;
      const float* th = st2;
      const float* tl = st2 + k * R;
      for (int j = 0; j < k; ++j) {
        const float b = __ldg(brow + j);
        dot2_add(s, c, b, th[j * R + lane]);
        sl = __fmaf_rn(b, tl[j * R + lane], sl);
      }
      bt = (double)s + (double)c + (double)sl;
    } else {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s = fma(__ldg(brow + j), st2[j * R + lane], s);
      bt = s;
    }
    Y[i * R + lane] = inv_s2 * (X[i * R + lane] - bt);
  }
}

// Z[i][r] = a W[i][r] + sum_j B[i][j] Tk[j][r]: a warp per row, lanes = columns,
// Tk staged in shared memory, FP64 accumulation
template <typename T>
__global__ void __launch_bounds__(256)
k_pc_affine(const T* __restrict__ B, const T* __restrict__ W, int64_t ldw,
            const double* __restrict__ Tk, int64_t n, int k, int nz, double a, T* __restrict__ Z,
            int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* st = reinterpret_cast<double*>(smem_raw);   // [k][nz]
  for (int e = threadIdx.x; e < k * nz; e += blockDim.x) st[e] = Tk[e];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  if (lane >= nz) return;
  for (int64_t i = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; i < n; i += (int64_t)gridDim.x * 8) {
    const T* brow = B + i * k;
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma((double)__ldg(brow + j), st[j * nz + lane], s);
    Z[i * ldz + lane] = (T)(a * (double)W[i * ldw + lane] + s);
  }
}

}  // namespace

void precond_free(Precond* pc) {
  if (!pc) return;
  cudaFree(pc->B);
  cudaFree(pc->Ginv);
  cudaFree(pc->partial);
  cudaFree(pc->t1);
  cudaFree(pc->t2);
  cudaFree(pc->xsplit);
  cudaFree(pc->Bd);
  *pc = Precond();
}

template <typename T>
agp_status caller_points(agp_plan_s* pl, CallerPoints<T>& cp, cudaStream_t st) {
  const int64_t n = pl->n;
  cp.st = st;
  cp.xo.assign(pl->P, nullptr);
  cp.wp.resize(pl->P);
  for (int s = 0; s < pl->P; ++s) {
    const Window& w = pl->win[s];
    AGP_CUDA(cudaMallocAsync(&cp.xo[s], sizeof(T) * n * w.d, st));
    k_unsort<T><<<nblk(n * w.d, 256), 256, 0, st>>>(reinterpret_cast<const T*>(w.xs), w.perm, n,
                                                    w.d, cp.xo[s]);
    cp.wp[s] = WinPts<T>{cp.xo[s], w.d};
  }
  return cuda_status(cudaGetLastError(), "caller_points");
}

template <typename T>
agp_status select_landmarks(agp_plan_s* pl, const CallerPoints<T>& cp, int k_req,
                            std::vector<int32_t>& all, cudaStream_t st) {
  const int64_t n = pl->n;
  const int P = pl->P;
  const int kw = std::max(1, (int)std::min<int64_t>(n, (k_req + P - 1) / P));
  const unsigned blocks = (unsigned)std::min<int64_t>(nblk(n, kFpsThreads), 1024);
  int32_t* chosen = nullptr;
  double* dist = nullptr;
  double* cand_d = nullptr;
  int64_t* cand_i = nullptr;
  AGP_CUDA(cudaMallocAsync(&chosen, sizeof(int32_t) * kw, st));
  AGP_CUDA(cudaMallocAsync(&dist, sizeof(double) * n, st));
  AGP_CUDA(cudaMallocAsync(&cand_d, sizeof(double) * blocks, st));
  AGP_CUDA(cudaMallocAsync(&cand_i, sizeof(int64_t) * blocks, st));
  all.clear();
  std::vector<int32_t> hk(kw);
  for (int s = 0; s < P; ++s) {
    AGP_CUDA(cudaMemsetAsync(chosen, 0, sizeof(int32_t) * kw, st));   // first landmark: point 0
    k_fill_double<<<nblk(n, 256), 256, 0, st>>>(dist, n, INFINITY);
    for (int step = 1; step < kw; ++step) {
      k_fps_dist<T><<<blocks, kFpsThreads, 0, st>>>(cp.xo[s], n, pl->win[s].d, chosen, step, dist,
                                                    cand_d, cand_i);
      k_fps_pick<<<1, kFpsThreads, 0, st>>>(cand_d, cand_i, (int)blocks, chosen, step);
    }
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(hk.data(), chosen, sizeof(int32_t) * kw, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    all.insert(all.end(), hk.begin(), hk.end());
  }
  cudaFreeAsync(chosen, st);
  cudaFreeAsync(dist, st);
  cudaFreeAsync(cand_d, st);
  cudaFreeAsync(cand_i, st);
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  return AGP_OK;
}

template <typename T>
agp_status precond_build(agp_plan_s* pl, int k_req, int rmax, Precond* pc, cudaStream_t st,
                         PrecondNlml* ex) {
  const int64_t n = pl->n;
  const int P = pl->P;
  if (!(pl->sigma_eps > 0)) return set_error(AGP_EINVAL, "the preconditioner needs sigma_eps > 0");
  CallerPoints<T> cp;
  AGP_TRY(caller_points<T>(pl, cp, st));
  std::vector<int32_t> all;
  AGP_TRY(select_landmarks<T>(pl, cp, k_req, all, st));
  const std::vector<WinPts<T>>& wp = cp.wp;
  const int k = (int)all.size();
  if (k > kMaxLandmarkSet)
    return set_error(AGP_EINVAL, "preconditioner: more than 512 landmarks after merging windows");
  int32_t* lm = nullptr;
  WinPts<T>* wpd = nullptr;
  AGP_CUDA(cudaMallocAsync(&lm, sizeof(int32_t) * k, st));
  AGP_CUDA(cudaMallocAsync(&wpd, sizeof(WinPts<T>) * P, st));
  AGP_CUDA(cudaMemcpyAsync(lm, all.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMemcpyAsync(wpd, wp.data(), sizeof(WinPts<T>) * P, cudaMemcpyHostToDevice, st));
  // B = K_{:,L}
  pc->k = k;
  pc->n = n;
  pc->rmax = rmax;
  pc->inv_s2 = 1.0 / (pl->sigma_eps * pl->sigma_eps);
  AGP_CUDA(cudaMalloc(&pc->B, sizeof(T) * n * k));
  k_kernel_cols<T><<<nblk(n * k, 256), 256, 0, st>>>(wpd, P, n, lm, k, pl->kernel, pl->ell,
                                                     pl->sigma_f * pl->sigma_f, 0, (T*)pc->B);
  // K_LL (FP64, exact kernel) + delta I and G = sigma_eps^2 K_LL + B^T B, then
  // Ginv by Cholesky. delta starts at 1e-6 sigma_f^2 P (1e-6 of the kernel's
  // diagonal value); when the FP64 Cholesky of G meets a non-positive pivot
  // (the landmarks outnumber the kernel's numerical rank and the columns of B
  // are numerically dependent) delta grows 100-fold and G is factorised
  // again, at most four times. delta is held fixed when M is differentiated.
  const double s2 = pl->sigma_eps * pl->sigma_eps;
  double *G = nullptr, *Li = nullptr, *KLL = nullptr, *KLL0 = nullptr, *BtB = nullptr;
  int* flag = nullptr;
  AGP_CUDA(cudaMallocAsync(&G, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&Li, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&KLL, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&KLL0, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&BtB, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&flag, sizeof(int), st));
  k_kernel_block<T><<<nblk((int64_t)k * k, 256), 256, 0, st>>>(
      wpd, P, n, lm, k, pl->kernel, pl->ell, pl->sigma_f * pl->sigma_f, 0, 0.0, KLL0);
  AGP_CUDA(cudaMemsetAsync(BtB, 0, sizeof(double) * k * k, st));
  const int64_t slices = std::min<int64_t>(64, (n + 4095) / 4096);
  const int64_t rps = (n + slices - 1) / slices;
  k_gram<T><<<dim3((k + 31) / 32, (k + 31) / 32, (unsigned)slices), 1024, 0, st>>>(
      (const T*)pc->B, (const T*)pc->B, n, k, rps, BtB);
  double delta = 1e-6 * pl->sigma_f * pl->sigma_f * P;
  int hflag = 1;
  for (int attempt = 0; attempt < 5 && hflag; ++attempt, delta *= 100.0) {
    AGP_CUDA(cudaMemcpyAsync(KLL, KLL0, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, st));
    k_shift_diag<<<nblk(k, 128), 128, 0, st>>>(KLL, k, delta);
    k_axpy<<<nblk((int64_t)k * k, 256), 256, 0, st>>>(KLL, s2, BtB, (int64_t)k * k, G);
    AGP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_cholesky<<<1, 1024, 0, st>>>(G, k, flag);
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    if (!hflag) break;
  }
  cudaFreeAsync(BtB, st);
  cudaFreeAsync(KLL0, st);
  k_tri_inverse<<<nblk(k, 128), 128, 0, st>>>(G, k, Li);
  AGP_CUDA(cudaMalloc(&pc->Ginv, sizeof(double) * k * k));
  k_gram_inverse<<<nblk((int64_t)k * k, 256), 256, 0, st>>>(Li, k, pc->Ginv);
  AGP_CUDA(cudaGetLastError());
  AGP_CUDA(cudaStreamSynchronize(st));
  if (ex && !hflag) {
    const size_t kk = (size_t)k * k;
    ex->delta = delta;
    std::vector<double> diag(k);
    double *dg = nullptr, *Kd = nullptr, *KLi = nullptr, *Kinv = nullptr, *W = nullptr;
    AGP_CUDA(cudaMallocAsync(&dg, sizeof(double) * k, st));
    AGP_CUDA(cudaMallocAsync(&Kd, sizeof(double) * kk, st));
    AGP_CUDA(cudaMallocAsync(&KLi, sizeof(double) * kk, st));
    AGP_CUDA(cudaMallocAsync(&Kinv, sizeof(double) * kk, st));
    AGP_CUDA(cudaMallocAsync(&W, sizeof(double) * kk, st));
    // log det G from its Cholesky factor (G now holds L)
    k_diag<<<nblk(k, 128), 128, 0, st>>>(G, k, dg);
    AGP_CUDA(cudaMemcpyAsync(diag.data(), dg, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    ex->Ginv.resize(kk);
    AGP_CUDA(cudaMemcpyAsync(ex->Ginv.data(), pc->Ginv, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    ex->logdet_G = 0.0;
    for (int j = 0; j < k; ++j) ex->logdet_G += 2.0 * std::log(diag[j]);
    // K_LL: Cholesky factor, inverse, log det
    AGP_CUDA(cudaMemcpyAsync(Kd, KLL, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st));
    ex->K.resize(kk);
    AGP_CUDA(cudaMemcpyAsync(ex->K.data(), Kd, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_cholesky<<<1, 1024, 0, st>>>(Kd, k, flag);
    k_tri_inverse<<<nblk(k, 128), 128, 0, st>>>(Kd, k, KLi);
    k_gram_inverse<<<nblk((int64_t)kk, 256), 256, 0, st>>>(KLi, k, Kinv);
    k_diag<<<nblk(k, 128), 128, 0, st>>>(Kd, k, dg);
    ex->Kchol.resize(kk);
    ex->Kinv.resize(kk);
    AGP_CUDA(cudaMemcpyAsync(ex->Kchol.data(), Kd, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemcpyAsync(ex->Kinv.data(), Kinv, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemcpyAsync(diag.data(), dg, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    // dB/dell, its landmark rows and B^T dB/dell
    AGP_CUDA(cudaMalloc(&pc->Bd, sizeof(T) * n * k));
    k_kernel_cols<T><<<nblk(n * k, 256), 256, 0, st>>>(wpd, P, n, lm, k, pl->kernel, pl->ell,
                                                       pl->sigma_f * pl->sigma_f, 1, (T*)pc->Bd);
    k_kernel_block<T><<<nblk((int64_t)kk, 256), 256, 0, st>>>(
        wpd, P, n, lm, k, pl->kernel, pl->ell, pl->sigma_f * pl->sigma_f, 1, 0.0, Kd);
    ex->Kder.resize(kk);
    AGP_CUDA(cudaMemcpyAsync(ex->Kder.data(), Kd, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * kk, st));
    k_gram<T><<<dim3((k + 31) / 32, (k + 31) / 32, (unsigned)slices), 1024, 0, st>>>(
        (const T*)pc->B, (const T*)pc->Bd, n, k, rps, W);
    ex->BtBder.resize(kk);
    AGP_CUDA(cudaMemcpyAsync(ex->BtBder.data(), W, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
    int kflag = 0;
    AGP_CUDA(cudaMemcpyAsync(&kflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaStreamSynchronize(st));
    for (void* q : {(void*)dg, (void*)Kd, (void*)KLi, (void*)Kinv, (void*)W}) cudaFreeAsync(q, st);
    if (kflag) {
      cudaFreeAsync(KLL, st);
      cudaFreeAsync(G, st);
      cudaFreeAsync(Li, st);
      cudaFreeAsync(flag, st);
      cudaFreeAsync(lm, st);
      cudaFreeAsync(wpd, st);
      return set_error(AGP_ENAN, "preconditioner: K_LL is not positive definite");
    }
    ex->logdet_K = 0.0;
    for (int j = 0; j < k; ++j) {
      ex->logdet_K += 2.0 * std::log(diag[j]);
      for (int b = j + 1; b < k; ++b) ex->Kchol[(size_t)j * k + b] = 0.0;   // keep the lower factor
    }
  }
  cudaFreeAsync(KLL, st);
  cudaFreeAsync(G, st);
  cudaFreeAsync(Li, st);
  cudaFreeAsync(flag, st);
  cudaFreeAsync(lm, st);
  cudaFreeAsync(wpd, st);
  if (hflag) return set_error(AGP_ENAN, "preconditioner: non-positive pivot in the Cholesky factor");
  // apply workspace
  pc->slices = (int)std::min<int64_t>(256, (n + 2047) / 2048);
  pc->rows_per_slice = (n + pc->slices - 1) / pc->slices;
  AGP_CUDA(cudaMalloc(&pc->partial, sizeof(double) * pc->slices * k * rmax));
  AGP_CUDA(cudaMalloc(&pc->t1, sizeof(double) * k * rmax));
  AGP_CUDA(cudaMalloc(&pc->t2, sizeof(T) * k * rmax * (sizeof(T) == 4 ? 2 : 1)));
  if (sizeof(T) == 4) AGP_CUDA(cudaMalloc(&pc->xsplit, sizeof(float) * 2 * n * rmax));
  return AGP_OK;
}

template <typename T>
agp_status precond_apply(const Precond& pc, const double* X, double* Y, int R, cudaStream_t st) {
  if (R > pc.rmax || R > 32) return set_error(AGP_EINVAL, "preconditioner: too many columns");
  const int k = pc.k;
  const float *xh = nullptr, *xl = nullptr;
  if (sizeof(T) == 4) {
    float* h = pc.xsplit;
    float* l = pc.xsplit + pc.n * R;
    k_split<<<nblk(pc.n * R, 256), 256, 0, st>>>(X, pc.n * R, h, l);
    xh = h;
    xl = l;
  }
  k_pc_bt<T><<<dim3((k + 31) / 32, pc.slices), 256, 0, st>>>((const T*)pc.B, X, xh, xl, pc.n, k, R,
                                                             pc.rows_per_slice, pc.partial);
  k_pc_mid<T><<<nblk((int64_t)k * R, 128), 128, 0, st>>>(pc.partial, pc.slices, pc.Ginv, k, R, 0,
                                                         pc.t1, pc.t2);
  k_pc_mid<T><<<nblk((int64_t)k * R, 128), 128, 0, st>>>(pc.partial, pc.slices, pc.Ginv, k, R, 1,
                                                         pc.t1, pc.t2);
  constexpr int NP = sizeof(T) == 4 ? 2 : 1;
  const size_t smem = sizeof(T) * NP * (size_t)k * R;
  AGP_CUDA(cudaFuncSetAttribute(k_pc_out<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(T) * NP * kMaxLandmarkSet * 32)));
  const unsigned blocks = (unsigned)std::min<int64_t>(nblk(pc.n, 8), 152 * 8);
  k_pc_out<T><<<blocks, 256, smem, st>>>((const T*)pc.B, X, pc.t2, pc.n, k, R, pc.inv_s2, Y);
  return cuda_status(cudaGetLastError(), "precond_apply");
}

template <typename T>
agp_status precond_bt(const Precond& pc, int der, const double* X, int R, double* out,
                      cudaStream_t st) {
  if (R > pc.rmax || R > 32) return set_error(AGP_EINVAL, "preconditioner: too many columns");
  if (der && !pc.Bd) return set_error(AGP_EINVAL, "preconditioner: no derivative columns");
  const int k = pc.k;
  const float *xh = nullptr, *xl = nullptr;
  if (sizeof(T) == 4) {
    float* h = pc.xsplit;
    float* l = pc.xsplit + pc.n * R;
    k_split<<<nblk(pc.n * R, 256), 256, 0, st>>>(X, pc.n * R, h, l);
    xh = h;
    xl = l;
  }
  k_pc_bt<T><<<dim3((k + 31) / 32, pc.slices), 256, 0, st>>>(
      (const T*)(der ? pc.Bd : pc.B), X, xh, xl, pc.n, k, R, pc.rows_per_slice, pc.partial);
  k_pc_mid<T><<<nblk((int64_t)k * R, 128), 128, 0, st>>>(pc.partial, pc.slices, pc.Ginv, k, R, 0,
                                                         pc.t1, pc.t2);
  AGP_CUDA(cudaGetLastError());
  AGP_CUDA(cudaMemcpyAsync(out, pc.t1, sizeof(double) * k * R, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  return AGP_OK;
}

template <typename T>
agp_status precond_affine(const Precond& pc, double a, const T* W, int64_t ldw, const double* Tk,
                          int nz, T* Z, int64_t ldz, cudaStream_t st) {
  if (nz < 1 || nz > 32) return set_error(AGP_EINVAL, "preconditioner: 1..32 columns");
  const size_t smem = sizeof(double) * (size_t)pc.k * nz;
  AGP_CUDA(cudaFuncSetAttribute(k_pc_affine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * kMaxLandmarkSet * 32)));
  const unsigned blocks = (unsigned)std::min<int64_t>(nblk(pc.n, 8), 152 * 8);
  k_pc_affine<T><<<blocks, 256, smem, st>>>((const T*)pc.B, W, ldw, Tk, pc.n, pc.k, nz, a, Z, ldz);
  return cuda_status(cudaGetLastError(), "precond_affine");
}

template <typename T>
agp_status precond_landmarks(agp_plan_s* pl, int k, std::vector<int32_t>& out, cudaStream_t st) {
  CallerPoints<T> cp;
  AGP_TRY(caller_points<T>(pl, cp, st));
  return select_landmarks<T>(pl, cp, k, out, st);
}

template agp_status caller_points<float>(agp_plan_s*, CallerPoints<float>&, cudaStream_t);
template agp_status caller_points<double>(agp_plan_s*, CallerPoints<double>&, cudaStream_t);
template agp_status select_landmarks<float>(agp_plan_s*, const CallerPoints<float>&, int,
                                            std::vector<int32_t>&, cudaStream_t);
template agp_status select_landmarks<double>(agp_plan_s*, const CallerPoints<double>&, int,
                                             std::vector<int32_t>&, cudaStream_t);
template agp_status precond_landmarks<float>(agp_plan_s*, int, std::vector<int32_t>&, cudaStream_t);
template agp_status precond_landmarks<double>(agp_plan_s*, int, std::vector<int32_t>&, cudaStream_t);
template agp_status precond_build<float>(agp_plan_s*, int, int, Precond*, cudaStream_t,
                                         PrecondNlml*);
template agp_status precond_build<double>(agp_plan_s*, int, int, Precond*, cudaStream_t,
                                          PrecondNlml*);
template agp_status precond_affine<float>(const Precond&, double, const float*, int64_t,
                                          const double*, int, float*, int64_t, cudaStream_t);
template agp_status precond_affine<double>(const Precond&, double, const double*, int64_t,
                                           const double*, int, double*, int64_t, cudaStream_t);
template agp_status precond_bt<float>(const Precond&, int, const double*, int, double*,
                                      cudaStream_t);
template agp_status precond_bt<double>(const Precond&, int, const double*, int, double*,
                                       cudaStream_t);
template agp_status precond_apply<float>(const Precond&, const double*, double*, int, cudaStream_t);
template agp_status precond_apply<double>(const Precond&, const double*, double*, int, cudaStream_t);

}  // namespace agp
