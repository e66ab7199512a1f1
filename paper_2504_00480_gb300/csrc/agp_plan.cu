// Plan construction and the C ABI of include/agp.h.
//
// Plan creation (once per point set):
//   a0  per window: grid-cell index floor(x_t n_os) of every point (exact:
//       n_os is a power of two), domain check x in [-1/4, 1/4)^d (Sec. 3.1),
//       counting sort of the points by cell, sorted coordinate copies, and
//       the list of work items (up to kItemPoints points of one cell each).
//   a1  per window: Fourier coefficients b_k of the kernel and of its
//       ell-derivative (Sec. 3.1 eq. (3.2), Sec. 3.2 eq. (3.4)) in FP64, and
//       the spectral multipliers b_k / prod_t (n_os psi_hat(k_t))^2 (Appendix A
//       deconvolution, applied once on each side of the transform pair).
// Matvec (Sec. 3.1 eq. (3.3), real part, then the weighted window sum):
//   out = sigma_eps^2 V; per block of RC right-hand sides: zero the grids,
//   spread, forward DFT, multiply, inverse DFT, interpolate (+= sigma_f^2 h).
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>

#include "agp_internal.cuh"

namespace agp {

namespace {
thread_local std::string g_last_error;
}

agp_status set_error(agp_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

agp_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return AGP_OK;
  if (e == cudaErrorMemoryAllocation)
    return set_error(AGP_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  return set_error(AGP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

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

constexpr int kErrTimeout = 2;      // error word bit: a bounded tensor-core wait expired

agp_status timeout_check(agp_plan_s* pl, cudaStream_t st) {
  int err = 0;
  AGP_CUDA(cudaMemcpyAsync(&err, pl->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  if (err & kErrTimeout) {
    const int keep = err & ~kErrTimeout;
    AGP_CUDA(cudaMemcpyAsync(pl->err_dev, &keep, sizeof(int), cudaMemcpyHostToDevice, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    return set_error(AGP_TIMEOUT, "a bounded wait in a tensor-core kernel expired");
  }
  return AGP_OK;
}

agp_status with_timeout_check(agp_plan_s* pl, agp_status s, cudaStream_t st) {
  if (s != AGP_OK && s != AGP_NOT_CONVERGED && s != AGP_ENAN) return s;
  const agp_status t = timeout_check(pl, st);
  return t == AGP_OK ? s : t;
}


namespace {

enum : int { kErrDomain = 1 };

// ---------------------------------------------------------------------------
// a0: binning and counting sort
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_bin_count(const T* __restrict__ X, int64_t ldx, int64_t n, int d, int f0, int f1,
                            int f2, int N, int n_os, int32_t* __restrict__ cell_of,
                            int32_t* __restrict__ counts, int* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int f[3] = {f0, f1, f2};
  int cell = 0;
  bool bad = false;
  for (int t = 0; t < d; ++t) {
    const T u = X[i * ldx + f[t]] * T(n_os);   // exact: n_os is a power of two
    const T fl = dev_floor(u);
    // cell coordinate c = floor(u) + N/2 must lie in [0, N)
    if (!(fl >= T(-N / 2) && fl < T(N / 2))) {
      bad = true;
    }
    int c = bad ? 0 : (int)fl + N / 2;
    cell = cell * N + c;
  }
  if (bad) {
    atomicOr(err, kErrDomain);
    cell = 0;
  }
  cell_of[i] = cell;
  atomicAdd(counts + cell, 1);
}

// Exclusive scan of `in` [n] into `out` [n + 1] by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_exclusive(const int32_t* __restrict__ in,
                                                         int32_t* __restrict__ out, int64_t n) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (n + 1023) / 1024;
  const int64_t a = tid * per, b = min(n, a + per);
  int64_t s = 0;
  for (int64_t i = a; i < b; ++i) s += in[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    out[n] = (int32_t)run;
  }
  __syncthreads();
  int64_t run = part[tid];
  for (int64_t i = a; i < b; ++i) {
    out[i] = (int32_t)run;
    run += in[i];
  }
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ X, int64_t ldx, int64_t n, int d, int f0, int f1,
                          int f2, const int32_t* __restrict__ cell_of,
                          const int32_t* __restrict__ cell_start, int32_t* __restrict__ fill,
                          int32_t* __restrict__ perm, T* __restrict__ xs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cell = cell_of[i];
  const int64_t pos = cell_start[cell] + atomicAdd(fill + cell, 1);
  perm[pos] = (int32_t)i;
  const int f[3] = {f0, f1, f2};
  for (int t = 0; t < d; ++t) xs[t * n + pos] = X[i * ldx + f[t]];
}

__global__ void k_chunks_per_cell(const int32_t* __restrict__ cell_start, int64_t cells, int cap,
                                  int32_t* __restrict__ nchunks) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const int cnt = cell_start[c + 1] - cell_start[c];
  nchunks[c] = (cnt + cap - 1) / cap;
}

__global__ void k_make_items(const int32_t* __restrict__ cell_start,
                             const int32_t* __restrict__ chunk_start, int64_t cells, int window,
                             int cap, int4* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const int a = cell_start[c], b = cell_start[c + 1];
  int o = chunk_start[c];
  for (int s = a; s < b; s += cap) items[o++] = make_int4(window, (int)c, s, min(cap, b - s));
}

// bins of every point in the caller's order: floor(x_t n_os) (a signed index)
template <typename T>
__global__ void k_bins_out(const T* __restrict__ xs, const int32_t* __restrict__ perm, int64_t n,
                           int d, int n_os, int32_t* __restrict__ bins) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int64_t i = perm[j];
  for (int t = 0; t < d; ++t) bins[i * d + t] = (int32_t)dev_floor(xs[t * n + j] * T(n_os));
}

// ---------------------------------------------------------------------------
// a1: Fourier coefficients (FP64)
// ---------------------------------------------------------------------------
// ---- outer boundary smoothing of kappa_R (Sec. 3.1) ----
// kappa_R(r) = kappa(r) for r <= a = 1/2 - eps, T(r) on the layer a < r < 1/2
// and kappa(1/2) beyond, with T the two-point Taylor polynomial of degree
// 2p - 1: T^(j)(a) = kappa^(j)(a), T(1/2) = kappa(1/2), T^(j)(1/2) = 0 for
// 1 <= j < p. The derivative kernel is regularised the same way (the
// construction is linear in the end data, so this is d kappa_R / d ell).
//
// The Taylor coefficients of kappa at a come from truncated power series
// arithmetic ("jets") in t = r - a: every kernel is a composition of +, *,
// 1/x, sqrt, exp and sin/cos, each with a standard recurrence for its
// series coefficients.
namespace jet {
__device__ void mul(const double* x, const double* y, double* z, int p) {
  double o[kBndMaxP];
  for (int k = 0; k < p; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += x[j] * y[k - j];
    o[k] = acc;
  }
  for (int k = 0; k < p; ++k) z[k] = o[k];
}
__device__ void scale(const double* x, double c, double* z, int p) {
  for (int k = 0; k < p; ++k) z[k] = c * x[k];
}
__device__ void exp_(const double* x, double* g, int p) {   // g' = x' g
  double o[kBndMaxP];
  o[0] = exp(x[0]);
  for (int k = 1; k < p; ++k) {
    double acc = 0.0;
    for (int j = 1; j <= k; ++j) acc += j * x[j] * o[k - j];
    o[k] = acc / k;
  }
  for (int k = 0; k < p; ++k) g[k] = o[k];
}
__device__ void recip(const double* x, double* g, int p) {  // x g = 1
  double o[kBndMaxP];
  o[0] = 1.0 / x[0];
  for (int k = 1; k < p; ++k) {
    double acc = 0.0;
    for (int j = 1; j <= k; ++j) acc += x[j] * o[k - j];
    o[k] = -acc * o[0];
  }
  for (int k = 0; k < p; ++k) g[k] = o[k];
}
__device__ void sqrt_(const double* x, double* g, int p) {  // g g = x
  double o[kBndMaxP];
  o[0] = sqrt(x[0]);
  for (int k = 1; k < p; ++k) {
    double acc = x[k];
    for (int j = 1; j < k; ++j) acc -= o[j] * o[k - j];
    o[k] = acc / (2.0 * o[0]);
  }
  for (int k = 0; k < p; ++k) g[k] = o[k];
}
__device__ void sincos_(const double* x, double* sn, double* cs, int p) {  // sn' = x' cs, cs' = -x' sn
  sn[0] = sin(x[0]);
  cs[0] = cos(x[0]);
  for (int k = 1; k < p; ++k) {
    double a = 0.0, b = 0.0;
    for (int j = 1; j <= k; ++j) {
      a += j * x[j] * cs[k - j];
      b += j * x[j] * sn[k - j];
    }
    sn[k] = a / k;
    cs[k] = -b / k;
  }
}
}  // namespace jet

// Taylor coefficients kappa^(j)(a) / j! (or of the ell-derivative), j < p.
__device__ void kernel_jet(int kernel, double a, double ell, int der, int p, double* f) {
  double r[kBndMaxP] = {0}, r2[kBndMaxP], t[kBndMaxP], u[kBndMaxP];
  r[0] = a;
  if (p > 1) r[1] = 1.0;
  jet::mul(r, r, r2, p);
  const double il = 1.0 / ell, il3 = il * il * il;
  if (kernel == AGP_GAUSS) {                 // exp(-r^2 / (2 ell^2)); der r^2/ell^3 kappa
    jet::scale(r2, -0.5 * il * il, t, p);
    jet::exp_(t, f, p);
    if (der) { jet::mul(f, r2, f, p); jet::scale(f, il3, f, p); }
  } else if (kernel == AGP_MATERN12) {       // exp(-r/ell); der r/ell^2 kappa
    jet::scale(r, -il, t, p);
    jet::exp_(t, f, p);
    if (der) { jet::mul(f, r, f, p); jet::scale(f, il * il, f, p); }
  } else if (kernel == AGP_MATERN32) {       // (1 + r/ell) exp(-r/ell); der r^2/ell^3 exp(-r/ell)
    jet::scale(r, -il, t, p);
    jet::exp_(t, u, p);
    if (der) {
      jet::mul(u, r2, f, p);
      jet::scale(f, il3, f, p);
    } else {
      jet::scale(r, il, t, p);
      t[0] += 1.0;
      jet::mul(t, u, f, p);
    }
  } else if (kernel == AGP_IMQ) {            // q = 1/(1 + r^2/ell^2), sqrt(q); der r^2/ell^3 sqrt(q) q
    jet::scale(r2, il * il, t, p);
    t[0] += 1.0;
    jet::recip(t, u, p);                     // q
    jet::sqrt_(u, f, p);
    if (der) { jet::mul(f, u, f, p); jet::mul(f, r2, f, p); jet::scale(f, il3, f, p); }
  } else {                                   // sinc: sin(w)/w, w = r/ell; der (sin(w)/w - cos(w))/ell
    double sn[kBndMaxP], cs[kBndMaxP];
    jet::scale(r, il, t, p);
    jet::sincos_(t, sn, cs, p);
    jet::recip(t, u, p);
    jet::mul(sn, u, f, p);
    if (der) for (int k = 0; k < p; ++k) f[k] = (f[k] - cs[k]) * il;
  }
}

// poly[der][j] = kappa^(j)(a)/j! eps^j (j < p, the Taylor data at the inner
// end in s = (r - a) / eps) and poly[der][2 kBndMaxP] = kappa(1/2). One
// thread per der.
__global__ void k_boundary_poly(double* __restrict__ poly, int kernel, double ell, double eps,
                                int p) {
  const int der = threadIdx.x;
  if (der > 1) return;
  double* e = poly + der * kBndStride;
  double f[kBndMaxP];
  kernel_jet(kernel, 0.5 - eps, ell, der, p, f);
  double pw = 1.0;
  for (int j = 0; j < p; ++j, pw *= eps) e[j] = f[j] * pw;
  e[2 * kBndMaxP] = kernel_value(kernel, 0.25, ell, der);
}

// The two-point Taylor polynomial on s in [0, 1] with Taylor data f_j at
// s = 0, value g at s = 1 and vanishing derivatives 1..p-1 there, in the
// two-point Taylor (Hermite) basis, which needs no linear solve:
//   T(s) = (1-s)^p sum_{j<p} f_j s^j sum_{k<p-j} C(p+k-1, k) s^k
//        + g s^p sum_{k<p} C(p+k-1, k) (1-s)^k.
__device__ double boundary_eval(const double* __restrict__ c, int p, double sl) {
  const double u = 1.0 - sl;
  double acc = 0.0, sj = 1.0;
  for (int j = 0; j < p; ++j, sj *= sl) {
    double sum = 0.0, bin = 1.0, sk = 1.0;          // bin = C(p+k-1, k)
    for (int k = 0; k < p - j; ++k) {
      sum += bin * sk;
      sk *= sl;
      bin = bin * (p + k) / (k + 1);
    }
    acc += c[j] * sj * sum;
  }
  double up = 1.0, sp = 1.0;
  for (int k = 0; k < p; ++k) { up *= u; sp *= sl; }
  double tail = 0.0, bin = 1.0, uk = 1.0;
  for (int k = 0; k < p; ++k) {
    tail += bin * uk;
    uk *= u;
    bin = bin * (p + k) / (k + 1);
  }
  return up * acc + c[2 * kBndMaxP] * sp * tail;
}

// samples[l] = kappa_R(|l / N|) (or its ell-derivative), l in I_N^d row-major,
// for coefficient job blockIdx.y; with p > 0 the outer boundary of kappa_R is
// smoothed by `poly`.
__global__ void k_kernel_samples(const CoefJob* __restrict__ jobs, int kernel, double ell,
                                 double eps, int p, const double* __restrict__ poly) {
  const CoefJob& jb = jobs[blockIdx.y];
  const int N = jb.N, d = jb.d, der = jb.der;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= jb.cells) return;
  int64_t rem = e;
  double r2 = 0.0;
  for (int t = d - 1; t >= 0; --t) {
    const int l = (int)(rem % N) - N / 2;
    rem /= N;
    const double x = (double)l / N;
    r2 += x * x;
  }
  double* out = jb.s0;
  if (p > 0) {
    const double* c = poly + der * kBndStride;
    const double r = sqrt(r2), a = 0.5 - eps;
    if (r >= 0.5) { out[e] = c[2 * kBndMaxP]; return; }
    if (r > a) {
      out[e] = boundary_eval(c, p, (r - a) / eps);
      return;
    }
  }
  out[e] = kernel_value(kernel, r2, ell, der);
}

// Largest squared norm of a window's (sorted) points, as the bit pattern of a
// non-negative double (monotone in the value), for the smoothing's domain.
template <typename T>
__global__ void k_max_norm2(const T* __restrict__ xs, int64_t n, int d,
                            unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double r2 = 0.0;
    for (int t = 0; t < d; ++t) {
      const double x = (double)xs[t * n + j];
      r2 += x * x;
    }
    m = fmax(m, r2);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// One axis of the d-dimensional DFT of eq. (3.2). The samples are real and
// even in every coordinate (kappa depends on |r| and the sample at
// l_t = -N/2 multiplies exp(i pi k_t) = (-1)^k_t), so the transform along each
// axis is the cosine sum sum_l in[l] costab[k][l], costab = cos(2 pi l k / N) / N
// (indices shifted by N/2), precomputed once per plan.
// Job blockIdx.y's axes alternate between its two scratch arrays and end in
// its b: axis 0 reads s0, odd axes read s1 and even axes s0.
__global__ void k_cos_axis(const CoefJob* __restrict__ jobs, int axis) {
  const CoefJob& jb = jobs[blockIdx.y];
  const int N = jb.N, d = jb.d;
  if (axis >= d) return;
  const double* __restrict__ in = (axis & 1) ? jb.s1 : jb.s0;
  double* __restrict__ out = (axis == d - 1) ? jb.b : ((axis & 1) ? jb.s0 : jb.s1);
  const double* __restrict__ costab = jb.costab;
  int64_t stride = 1;
  for (int t = d - 1; t > axis; --t) stride *= N;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= jb.cells) return;
  const int kk = (int)((e / stride) % N);
  const int64_t base = e - (int64_t)kk * stride;
  const double* row = costab + (int64_t)kk * N;
  double s = 0.0;
  for (int li = 0; li < N; ++li) s += in[base + (int64_t)li * stride] * row[li];
  out[e] = s;
}

// Kaiser-Bessel values of every (sorted) point, psi(frac(u_t) + s - 1 - tap)
// for tap < 2s, where u_t = x_t n_os (Appendix A window in grid units,
// divided by I0(b s)); evaluated in FP64 and rounded to the plan precision.
// Layout per point (window_wpp values): dimensions 0..d-2 as ttp values each
// (zero padded), then the last dimension's taps each written twice.
template <typename T>
__global__ void k_window_values(const T* __restrict__ xs, int64_t n, int d, int n_os, int s,
                                int ttp, double b, double norm, T* __restrict__ wts) {
  const int wpp = (d - 1) * ttp + 4 * s;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * wpp) return;
  const int64_t j = e / wpp;
  const int o = (int)(e - j * wpp);
  int t, tap;
  if (o < (d - 1) * ttp) {
    t = o / ttp;
    tap = o - t * ttp;
  } else {
    t = d - 1;
    tap = (o - (d - 1) * ttp) / 2;
  }
  double v = 0.0;
  if (tap < 2 * s) {
    const double u = (double)xs[(int64_t)t * n + j] * n_os;   // exact: n_os is a power of two
    const double delta = (u - floor(u)) + (double)(s - 1 - tap);
    v = kb_psi(delta, (double)s, b, norm);
  }
  wts[e] = (T)v;
}

// Spectral multiplier on the half-spectrum layout [K]^(d-1) x [Kh]:
//   D(k) = w(k) b_{|k|} / prod_t winhat(k_t)^2,
//   w(k) = (1[k in I_N] + 1[-k in I_N]) / 2,
// the real-part symmetrisation of eq. (3.3) over the asymmetric I_N.
template <typename T>
__global__ void k_build_dmul(const CoefJob* __restrict__ jobs) {
  const CoefJob& jb = jobs[blockIdx.y];
  const int N = jb.N, d = jb.d;
  const double* __restrict__ b = jb.b;
  const double* __restrict__ winhat = jb.winhat;
  T* __restrict__ dmul = reinterpret_cast<T*>(jb.dmul);
  const int K = N + 1, Kh = N / 2 + 1;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= jb.dmul_elems) return;
  int k[3];
  int64_t rem = e;
  k[d - 1] = (int)(rem % Kh);
  rem /= Kh;
  for (int t = d - 2; t >= 0; --t) {
    k[t] = (int)(rem % K) - N / 2;
    rem /= K;
  }
  bool in_pos = true, in_neg = true;
  int64_t bidx = 0;
  double den = 1.0;
  for (int t = 0; t < d; ++t) {
    const int kt = k[t];
    in_pos = in_pos && (kt >= -N / 2) && (kt <= N / 2 - 1);
    in_neg = in_neg && (-kt >= -N / 2) && (-kt <= N / 2 - 1);
    const int ka = kt < 0 ? -kt : kt;
    const int bi = (ka == N / 2) ? 0 : ka + N / 2;   // b is even and N-periodic
    bidx = bidx * N + bi;
    const double wh = winhat[kt + N / 2];
    den *= wh * wh;
  }
  const double wgt = 0.5 * ((in_pos ? 1.0 : 0.0) + (in_neg ? 1.0 : 0.0));
  dmul[e] = (T)(wgt * b[bidx] / den);
}

// Half spectrum (forward-DFT layout) -> full I_N^d spectrum divided by the
// window transform: chat[r][k] = X(k) / prod_t winhat(k_t), with
// X(k) = conj(X(-k)) for k_d < 0.
template <typename T, typename T2>
__global__ void k_extract_spectrum(const T2* __restrict__ spec, const double* __restrict__ winhat,
                                   int N, int d, int RC, int R, T2* __restrict__ out) {
  const int K = N + 1, Kh = N / 2 + 1;
  int64_t cells = 1;
  for (int t = 0; t < d; ++t) cells *= N;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cells * R) return;
  const int r = (int)(e / cells);
  int64_t rem = e - (int64_t)r * cells;
  int k[3];
  for (int t = d - 1; t >= 0; --t) {
    k[t] = (int)(rem % N) - N / 2;
    rem /= N;
  }
  const bool conj = k[d - 1] < 0;
  int64_t si = 0;
  double den = 1.0;
  for (int t = 0; t < d; ++t) {
    const int kk = conj ? -k[t] : k[t];
    si = (t == d - 1) ? si * Kh + kk : si * K + (kk + N / 2);
    den *= winhat[k[t] + N / 2];
  }
  T2 v = spec[si * RC + r];
  if (conj) v.y = -v.y;
  v.x = (T)(v.x / den);
  v.y = (T)(v.y / den);
  out[e] = v;
}

// Full spectrum fhat[r][k] on I_N^d -> Hermitian half layout for the inverse
// DFT: X(k) = (F(k) + conj(F(-k))) / 2, F(k) = fhat(k) / prod winhat(k_t)
// (zero outside I_N), k in [-N/2, N/2]^(d-1) x [0, N/2].
template <typename T, typename T2>
__global__ void k_insert_spectrum(const T2* __restrict__ fhat, const double* __restrict__ winhat,
                                  int N, int d, int RC, int R, T2* __restrict__ spec) {
  const int K = N + 1, Kh = N / 2 + 1;
  int64_t total = Kh;
  for (int t = 0; t < d - 1; ++t) total *= K;
  int64_t cells = 1;
  for (int t = 0; t < d; ++t) cells *= N;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total * RC) return;
  const int r = (int)(e % RC);
  int64_t rem = e / RC;
  int k[3];
  k[d - 1] = (int)(rem % Kh);
  rem /= Kh;
  for (int t = d - 2; t >= 0; --t) {
    k[t] = (int)(rem % K) - N / 2;
    rem /= K;
  }
  T2 out;
  out.x = out.y = T(0);
  if (r < R) {
    double den = 1.0;
    bool in_pos = true, in_neg = true;
    int64_t ip = 0, ineg = 0;
    for (int t = 0; t < d; ++t) {
      in_pos = in_pos && k[t] <= N / 2 - 1;
      in_neg = in_neg && -k[t] <= N / 2 - 1;
      ip = ip * N + (k[t] + N / 2);
      ineg = ineg * N + (-k[t] + N / 2);
      den *= winhat[k[t] + N / 2];
    }
    double re = 0.0, im = 0.0;
    if (in_pos) {
      const T2 f = fhat[(int64_t)r * cells + ip];
      re += f.x;
      im += f.y;
    }
    if (in_neg) {
      const T2 f = fhat[(int64_t)r * cells + ineg];
      re += f.x;
      im -= f.y;
    }
    out.x = (T)(0.5 * re / den);
    out.y = (T)(0.5 * im / den);
  }
  spec[e] = out;
}

template <typename T>
__global__ void k_init_out(T* __restrict__ Out, int64_t ldo, const T* __restrict__ V, int64_t ldv,
                           int64_t n, int R, T alpha) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t i = e / R;
  const int r = (int)(e - i * R);
  Out[i * ldo + r] = (alpha == T(0)) ? T(0) : alpha * V[i * ldv + r];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Modified Bessel function I0 by its power series sum_j ((x/2)^2)^j / (j!)^2
// (all terms positive, so it converges without cancellation).
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int j = 1; j < 500; ++j) {
    term *= q / ((double)j * (double)j);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

size_t elem_size(agp_prec p) { return p == AGP_F64 ? 8 : 4; }

agp_status validate(const agp_plan_desc* d) {
  if (!d) return set_error(AGP_EINVAL, "desc is NULL");
  if (d->n < 1 || d->n > (int64_t)INT32_MAX - 1) return set_error(AGP_EINVAL, "n out of range");
  if (d->p < 1 || !d->X || d->ldx < d->p) return set_error(AGP_EINVAL, "bad X / p / ldx");
  if (d->P < 1 || d->P > kMaxWindows || !d->win_ptr || !d->win_feat || !d->N)
    return set_error(AGP_EINVAL, "bad windows");
  if (d->sigma_os != 2) return set_error(AGP_EINVAL, "sigma_os must be 2");
  if (d->cutoff < 2 || d->cutoff > 6) return set_error(AGP_EINVAL, "cutoff must be in [2, 6]");
  if (!(d->ell > 0) || !std::isfinite(d->ell) || !std::isfinite(d->sigma_f) ||
      !std::isfinite(d->sigma_eps))
    return set_error(AGP_EINVAL, "bad hyperparameters");
  if (d->kernel < AGP_GAUSS || d->kernel > AGP_SINC)
    return set_error(AGP_EINVAL, "bad kernel");
  if (d->prec != AGP_F32 && d->prec != AGP_F64) return set_error(AGP_EINVAL, "bad prec");
  std::vector<int> used(d->p, 0);
  if (d->win_ptr[0] != 0) return set_error(AGP_EINVAL, "win_ptr[0] must be 0");
  for (int s = 0; s < d->P; ++s) {
    const int a = d->win_ptr[s], b = d->win_ptr[s + 1];
    if (b - a < 1 || b - a > kMaxDim) return set_error(AGP_EINVAL, "window dimension must be 1..3");
    const int N = d->N[s];
    if (N != 8 && N != 16 && N != 32 && N != 64) return set_error(AGP_EINVAL, "N must be 8, 16, 32 or 64");
    if (d->cutoff > N / 2) return set_error(AGP_EINVAL, "cutoff must be <= N/2");
    for (int q = a; q < b; ++q) {
      const int f = d->win_feat[q];
      if (f < 0 || f >= d->p) return set_error(AGP_EINVAL, "feature id out of range");
      if (used[f]++) return set_error(AGP_EINVAL, "windows must be disjoint");
    }
  }
  return AGP_OK;
}

// The coefficient jobs of a plan (window s, der) -> 2 s + der, with their
// scratch arrays; built once, the buffers they point to never move.
agp_status build_coef_jobs(agp_plan_s* pl) {
  std::vector<CoefJob> jobs;
  int64_t scratch = 0;
  for (const Window& w : pl->win) scratch += 4 * w.cells;
  AGP_CUDA(cudaMalloc(&pl->coef_scratch, sizeof(double) * scratch));
  double* sp = pl->coef_scratch;
  for (Window& w : pl->win)
    for (int der = 0; der < 2; ++der) {
      CoefJob jb;
      jb.s0 = sp;
      jb.s1 = sp + w.cells;
      sp += 2 * w.cells;
      jb.b = der ? w.bder : w.b;
      jb.costab = w.costab;
      jb.winhat = reinterpret_cast<const double*>(w.winhat);
      jb.dmul = der ? w.dmul_der : w.dmul;
      jb.N = w.N;
      jb.d = w.d;
      jb.der = der;
      jb.cells = w.cells;
      jb.dmul_elems = w.dmul_elems;
      jobs.push_back(jb);
      pl->coef_cells_max = std::max(pl->coef_cells_max, w.cells);
      pl->coef_dmul_max = std::max(pl->coef_dmul_max, w.dmul_elems);
      pl->coef_dmax = std::max(pl->coef_dmax, w.d);
    }
  AGP_CUDA(cudaMalloc(&pl->coef_jobs, sizeof(CoefJob) * jobs.size()));
  AGP_CUDA(cudaMemcpy(pl->coef_jobs, jobs.data(), sizeof(CoefJob) * jobs.size(),
                      cudaMemcpyHostToDevice));
  pl->n_coef_jobs = (int)jobs.size();
  return AGP_OK;
}

// a1 for every window and both coefficient sets: one launch per stage
// (samples, each DFT axis, multipliers), the jobs along gridDim.y.
template <typename T>
agp_status compute_coeffs(agp_plan_s* pl, cudaStream_t st) {
  if (!pl->coef_jobs) AGP_TRY(build_coef_jobs(pl));
  if (pl->bnd_p > 0)
    k_boundary_poly<<<1, 32, 0, st>>>(pl->bnd_poly, pl->kernel, pl->ell, pl->bnd_eps, pl->bnd_p);
  const dim3 gs(nblk(pl->coef_cells_max, 256), pl->n_coef_jobs);
  k_kernel_samples<<<gs, 256, 0, st>>>(pl->coef_jobs, pl->kernel, pl->ell, pl->bnd_eps,
                                       pl->bnd_p, pl->bnd_poly);
  for (int axis = 0; axis < pl->coef_dmax; ++axis)
    k_cos_axis<<<gs, 256, 0, st>>>(pl->coef_jobs, axis);
  const dim3 gm(nblk(pl->coef_dmul_max, 256), pl->n_coef_jobs);
  k_build_dmul<T><<<gm, 256, 0, st>>>(pl->coef_jobs);
  AGP_CUDA(cudaGetLastError());
  return AGP_OK;
}

void free_plan(agp_plan_s* pl) {
  if (!pl) return;
  for (auto& w : pl->win) {
    cudaFree(w.perm);
    cudaFree(w.xs);
    cudaFree(w.wts);
    cudaFree(w.costab);
    cudaFree(w.cell_start);
    cudaFree(w.b);
    cudaFree(w.bder);
    cudaFree(w.dmul);
    cudaFree(w.dmul_der);
    cudaFree(w.winhat);
    cudaFree(w.tw);
    cudaFree(w.grid);
    cudaFree(w.specA);
    cudaFree(w.specB);
    cudaFree(w.fft_self);
  }
  for (auto& g : pl->groups) cudaFree(g.tab);
  for (auto& e : pl->prof_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  cudaFree(pl->items_all);
  cudaFree(pl->runs3);
  cudaFree(pl->wins_dev);
  cudaFree(pl->grid_maps);
  cudaFree(pl->err_dev);
  if (pl->side) cudaStreamDestroy(pl->side);
  if (pl->fork_ev) cudaEventDestroy(pl->fork_ev);
  if (pl->join_ev) cudaEventDestroy(pl->join_ev);
  cudaFree(pl->bnd_poly);
  cudaFree(pl->coef_jobs);
  cudaFree(pl->coef_scratch);
  delete pl;
}

// (Re)build the work items of every window with at most `cap` points each,
// grouped by window dimension (all windows of one d share a launch).
agp_status build_items(agp_plan_s* pl, int cap, cudaStream_t st) {
  std::vector<int64_t> n_items(pl->P, 0);
  std::vector<int32_t*> chunk_start(pl->P, nullptr);
  struct Free {
    std::vector<int32_t*>& v;
    cudaStream_t st;
    ~Free() {
      for (auto* p : v)
        if (p) cudaFreeAsync(p, st);
    }
  } fr{chunk_start, st};
  for (int s = 0; s < pl->P; ++s) {
    Window& w = pl->win[s];
    int32_t* nch = nullptr;
    AGP_CUDA(cudaMallocAsync(&nch, sizeof(int32_t) * w.cells, st));
    AGP_CUDA(cudaMallocAsync(&chunk_start[s], sizeof(int32_t) * (w.cells + 1), st));
    k_chunks_per_cell<<<nblk(w.cells, 256), 256, 0, st>>>(w.cell_start, w.cells, cap, nch);
    k_scan_exclusive<<<1, 1024, 0, st>>>(nch, chunk_start[s], w.cells);
    AGP_CUDA(cudaGetLastError());
    int32_t tot = 0;
    AGP_CUDA(cudaMemcpyAsync(&tot, chunk_start[s] + w.cells, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    AGP_CUDA(cudaFreeAsync(nch, st));
    n_items[s] = tot;
  }
  int64_t total = 0;
  for (int s = 0; s < pl->P; ++s) total += n_items[s];
  int4* items = nullptr;
  AGP_CUDA(cudaMalloc(&items, sizeof(int4) * (total > 0 ? total : 1)));
  int64_t off = 0;
  for (int dd = 1; dd <= kMaxDim; ++dd) {
    pl->items_by_d[dd - 1] = off;
    for (int s = 0; s < pl->P; ++s) {
      Window& w = pl->win[s];
      if (w.d != dd) continue;
      w.items = items + off;
      w.n_items = n_items[s];
      k_make_items<<<nblk(w.cells, 256), 256, 0, st>>>(w.cell_start, chunk_start[s], w.cells, s,
                                                       cap, w.items);
      off += n_items[s];
    }
  }
  pl->items_by_d[kMaxDim] = off;
  AGP_CUDA(cudaGetLastError());
  AGP_CUDA(cudaStreamSynchronize(st));
  if (pl->items_all) cudaFree(pl->items_all);
  pl->items_all = items;
  pl->item_points = cap;
  // runs of kRunCells cells along the last dimension for the tensor-core
  // kernels (host: cell_start of every d = 3 window, the non-empty runs)
  if (!pl->runs3) {
    std::vector<int4> runs;
    for (int s = 0; s < pl->P; ++s) {
      const Window& w = pl->win[s];
      if (w.d != 3 || w.N % kRunCells != 0) continue;
      std::vector<int32_t> cs(w.cells + 1);
      AGP_CUDA(cudaMemcpyAsync(cs.data(), w.cell_start, sizeof(int32_t) * (w.cells + 1),
                               cudaMemcpyDeviceToHost, st));
      AGP_CUDA(cudaStreamSynchronize(st));
      for (int64_t c = 0; c < w.cells; c += kRunCells) {
        const int a = cs[c], b = cs[c + kRunCells];
        for (int q = a; q < b; q += kRunPoints)
          runs.push_back(make_int4(s | (kRunCells << 16), (int)c, q, std::min(kRunPoints, b - q)));
      }
    }
    pl->n_runs3 = (int64_t)runs.size();
    if (!runs.empty()) {
      AGP_CUDA(cudaMalloc(&pl->runs3, sizeof(int4) * runs.size()));
      AGP_CUDA(cudaMemcpyAsync(pl->runs3, runs.data(), sizeof(int4) * runs.size(),
                               cudaMemcpyHostToDevice, st));
      AGP_CUDA(cudaStreamSynchronize(st));
    }
  }
  return AGP_OK;
}

template <typename T>
agp_status plan_build(agp_plan_s* pl, const agp_plan_desc* d, cudaStream_t st) {
  const int64_t n = pl->n;
  const T* X = reinterpret_cast<const T*>(d->X);
  AGP_CUDA(cudaMalloc(&pl->err_dev, sizeof(int) * 4));
  AGP_CUDA(cudaMemsetAsync(pl->err_dev, 0, sizeof(int) * 4, st));

  int32_t* cell_of = nullptr;
  AGP_CUDA(cudaMallocAsync(&cell_of, sizeof(int32_t) * n, st));

  for (int s = 0; s < pl->P; ++s) {
    Window& w = pl->win[s];
    int32_t *counts = nullptr, *fill = nullptr;
    AGP_CUDA(cudaMalloc(&w.perm, sizeof(int32_t) * n));
    AGP_CUDA(cudaMalloc(&w.xs, sizeof(T) * n * w.d));
    AGP_CUDA(cudaMalloc(&w.cell_start, sizeof(int32_t) * (w.cells + 1)));
    AGP_CUDA(cudaMallocAsync(&counts, sizeof(int32_t) * w.cells, st));
    AGP_CUDA(cudaMallocAsync(&fill, sizeof(int32_t) * w.cells, st));
    AGP_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * w.cells, st));
    AGP_CUDA(cudaMemsetAsync(fill, 0, sizeof(int32_t) * w.cells, st));
    k_bin_count<T><<<nblk(n, 256), 256, 0, st>>>(X, d->ldx, n, w.d, w.feat[0], w.feat[1],
                                                 w.feat[2], w.N, w.n_os, cell_of, counts,
                                                 pl->err_dev);
    k_scan_exclusive<<<1, 1024, 0, st>>>(counts, w.cell_start, w.cells);
    k_scatter<T><<<nblk(n, 256), 256, 0, st>>>(X, d->ldx, n, w.d, w.feat[0], w.feat[1],
                                               w.feat[2], cell_of, w.cell_start, fill, w.perm,
                                               reinterpret_cast<T*>(w.xs));
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaFreeAsync(counts, st));
    AGP_CUDA(cudaFreeAsync(fill, st));
  }
  int err = 0;
  AGP_CUDA(cudaMemcpyAsync(&err, pl->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  if (err & kErrDomain) {
    cudaFree(cell_of);
    return set_error(AGP_EDOMAIN, "a point lies outside [-1/4, 1/4)^d in some window");
  }

  AGP_CUDA(cudaFreeAsync(cell_of, st));
  AGP_TRY(build_items(pl, kItemPoints, st));

  // Deconvolution factors, twiddles, coefficient buffers, grids.
  std::vector<WinDev<T>> wd(pl->P);
  for (int s = 0; s < pl->P; ++s) {
    Window& w = pl->win[s];
    const double b = pl->kb_b;
    const double i0bs = bessel_i0(b * w.s);
    w.winhat_h.resize(w.K);
    for (int kk = 0; kk < w.K; ++kk) {
      const double k = kk - w.N / 2;
      const double om = 2.0 * M_PI * k / w.n_os;
      w.winhat_h[kk] = bessel_i0(w.s * std::sqrt(b * b - om * om)) / i0bs;
    }
    AGP_CUDA(cudaMalloc(&w.winhat, sizeof(double) * w.K));
    AGP_CUDA(cudaMemcpyAsync(w.winhat, w.winhat_h.data(), sizeof(double) * w.K,
                             cudaMemcpyHostToDevice, st));
    // twiddles exp(-2 pi i k (a + lo) / n_os), [K][W]
    const int lo = -w.N / 2 - w.s + 1;
    std::vector<T> tw(2 * (size_t)w.K * w.W);
    for (int kk = 0; kk < w.K; ++kk) {
      const int k = kk - w.N / 2;
      for (int a = 0; a < w.W; ++a) {
        // angle = -2 pi k l / n_os, reduced exactly modulo n_os in integers
        long long kl = (long long)k * (a + lo);
        kl %= w.n_os;
        if (kl < 0) kl += w.n_os;
        const double ang = -2.0 * M_PI * (double)kl / (double)w.n_os;
        tw[2 * ((size_t)kk * w.W + a)] = (T)std::cos(ang);
        tw[2 * ((size_t)kk * w.W + a) + 1] = (T)std::sin(ang);
      }
    }
    AGP_CUDA(cudaMalloc(&w.tw, sizeof(T) * tw.size()));
    AGP_CUDA(cudaMemcpyAsync(w.tw, tw.data(), sizeof(T) * tw.size(), cudaMemcpyHostToDevice, st));
    // cosine table of the coefficient DFT: cos(2 pi l k / N) / N, l, k in I_N
    std::vector<double> ct((size_t)w.N * w.N);
    for (int kk = 0; kk < w.N; ++kk)
      for (int li = 0; li < w.N; ++li) {
        long long lk = (long long)(kk - w.N / 2) * (li - w.N / 2);
        lk %= w.N;
        if (lk < 0) lk += w.N;
        ct[(size_t)kk * w.N + li] = std::cos(2.0 * M_PI * (double)lk / (double)w.N) / w.N;
      }
    AGP_CUDA(cudaMalloc(&w.costab, sizeof(double) * ct.size()));
    AGP_CUDA(cudaMemcpyAsync(w.costab, ct.data(), sizeof(double) * ct.size(),
                             cudaMemcpyHostToDevice, st));
    AGP_CUDA(cudaStreamSynchronize(st));   // host tables go out of scope
    // window values of every sorted point (they do not depend on the hyperparameters)
    const int ttp = window_ttp(w.s);
    const int wpp = window_wpp(w.d, w.s);
    AGP_CUDA(cudaMalloc(&w.wts, sizeof(T) * n * wpp));
    k_window_values<T><<<nblk(n * wpp, 256), 256, 0, st>>>(
        reinterpret_cast<const T*>(w.xs), n, w.d, w.n_os, w.s, ttp, pl->kb_b, pl->kb_norm,
        reinterpret_cast<T*>(w.wts));
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMalloc(&w.b, sizeof(double) * w.cells));
    AGP_CUDA(cudaMalloc(&w.bder, sizeof(double) * w.cells));
    AGP_CUDA(cudaMalloc(&w.dmul, sizeof(T) * w.dmul_elems));
    AGP_CUDA(cudaMalloc(&w.dmul_der, sizeof(T) * w.dmul_elems));
    AGP_CUDA(cudaMalloc(&w.grid, sizeof(T) * w.grid_elems * pl->rc_max));
    AGP_CUDA(cudaMalloc(&w.specA, 2 * sizeof(T) * w.spec_elems * pl->rc_max));
    AGP_CUDA(cudaMalloc(&w.specB, 2 * sizeof(T) * w.spec_elems * pl->rc_max));
    wd[s].xs = reinterpret_cast<const T*>(w.xs);
    wd[s].perm = w.perm;
    wd[s].wts = reinterpret_cast<const T*>(w.wts);
    wd[s].grid = reinterpret_cast<T*>(w.grid);
    wd[s].cell_start = w.cell_start;
    wd[s].n = n;
    wd[s].N = w.N;
    wd[s].n_os = w.n_os;
    wd[s].W = w.W;
  }
  AGP_CUDA(cudaMalloc(&pl->wins_dev, sizeof(WinDev<T>) * pl->P));
  AGP_CUDA(cudaMemcpyAsync(pl->wins_dev, wd.data(), sizeof(WinDev<T>) * pl->P,
                           cudaMemcpyHostToDevice, st));
  // FP32: tensor maps of the d = 3 grids for the tensor-memory spreading
  // kernel's bulk reductions (without them that kernel is not selected)
  if constexpr (std::is_same<T, float>::value) {
    std::vector<int> win_d(pl->P);
    bool any3 = false;
    for (int s = 0; s < pl->P; ++s) {
      win_d[s] = pl->win[s].d;
      any3 = any3 || win_d[s] == 3;
    }
    struct alignas(64) MapSlot {
      unsigned char b[kGridMapBytes];
    };
    std::vector<MapSlot> maps(2 * (size_t)pl->P);
    if (any3 && spread_tm_supported(3, pl->s, 32) &&
        encode_grid_maps(wd.data(), win_d.data(), pl->P, pl->s, maps.data())) {
      AGP_CUDA(cudaMalloc(&pl->grid_maps, sizeof(MapSlot) * maps.size()));
      AGP_CUDA(cudaMemcpyAsync(pl->grid_maps, maps.data(), sizeof(MapSlot) * maps.size(),
                               cudaMemcpyHostToDevice, st));
      AGP_CUDA(cudaStreamSynchronize(st));
    }
  }
  // DFT buffer tables: one per window, and one per (d, N) group of windows
  std::vector<FftWin> fw(pl->P);
  for (int s = 0; s < pl->P; ++s) {
    Window& w = pl->win[s];
    fw[s] = FftWin{w.grid, w.specA, w.specB, w.tw, w.dmul, w.dmul_der};
    AGP_CUDA(cudaMalloc(&w.fft_self, sizeof(FftWin)));
    AGP_CUDA(cudaMemcpyAsync(w.fft_self, &fw[s], sizeof(FftWin), cudaMemcpyHostToDevice, st));
  }
  std::vector<std::vector<FftWin>> gtab;
  for (int s = 0; s < pl->P; ++s) {
    const Window& w = pl->win[s];
    size_t gi = 0;
    while (gi < pl->groups.size() && !(pl->groups[gi].d == w.d && pl->groups[gi].N == w.N)) ++gi;
    if (gi == pl->groups.size()) {
      FftGroup g = w.self_group();
      g.count = 0;
      g.tab = nullptr;
      pl->groups.push_back(g);
      gtab.emplace_back();
    }
    pl->groups[gi].count += 1;
    gtab[gi].push_back(fw[s]);
  }
  for (size_t gi = 0; gi < pl->groups.size(); ++gi) {
    AGP_CUDA(cudaMalloc(&pl->groups[gi].tab, sizeof(FftWin) * gtab[gi].size()));
    AGP_CUDA(cudaMemcpyAsync(pl->groups[gi].tab, gtab[gi].data(), sizeof(FftWin) * gtab[gi].size(),
                             cudaMemcpyHostToDevice, st));
  }
  AGP_TRY(compute_coeffs<T>(pl, st));
  AGP_CUDA(cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking));
  AGP_CUDA(cudaEventCreateWithFlags(&pl->fork_ev, cudaEventDisableTiming));
  AGP_CUDA(cudaEventCreateWithFlags(&pl->join_ev, cudaEventDisableTiming));
  AGP_CUDA(cudaStreamSynchronize(st));   // host tables go out of scope
  return AGP_OK;
}

// Right-hand sides of the next pass for R remaining columns. With the
// tensor-core kernels on, FP32 plans with a d = 3 window that they support
// take 17 or more columns in a pass of 32 and 9 .. 16 columns in a pass of
// 16: a tensor-core pass costs about the same for any column count up to its
// width (a 17-column pass of 32 is still cheaper than the FMA kernels'
// 24-column pass, and than 16 columns plus a narrow FMA pass for the rest),
// and a 16-column pass saves half of the DFT work of a 32-column one.
int pick_rc(const agp_plan_s* pl, int R) {
  if (pl->use_tc && pl->prec == AGP_F32 && R >= 9) {
    for (const Window& w : pl->win)
      if (spread_tc_supported(w.d, pl->s, 32) && interp_tc_supported(w.d, pl->s, 32))
        return R >= 17 ? 32 : 16;
  }
  return rhs_block_width(pl->prec, R);
}

// Autotuner results, shared by the plans of a process: key (precision,
// cutoff, pass width, right-hand sides, window shapes, log2 n) -> the chosen
// kernel family, work-item size and its time per matvec.
struct TuneEntry {
  int mode, points;
  double ms;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;

// Kernel family of a pass's d = 3 spreading / interpolation (rc grid
// columns, Rc of them in use):
// 3 the persistent tensor-memory kernel over cell runs, 2 the shared-memory
// tensor-core kernel over cell runs, 1 the tensor-core kernel over work items
// where it supports the case, else 0, the FMA kernel over work items.
int spread_family3(const agp_plan_s* pl, int rc) {
  if (pl->prec != AGP_F32 || !pl->use_tc) return 0;
  if (pl->runs3 && pl->grid_maps && (pl->use_tc == 1 || pl->use_tc == 3) &&
      spread_tm_supported(3, pl->s, rc))
    return 3;
  if (pl->runs3 && spread_tc_supported(3, pl->s, rc)) return 2;
  return spread_tc_supported(3, pl->s, rc) ? 1 : 0;
}

int interp_family3(const agp_plan_s* pl, int rc, int Rc) {
  if (pl->prec != AGP_F32 || !pl->use_tc) return 0;
  if (pl->runs3 && pl->use_tc == 3 && interp_tm_supported(3, pl->s, rc, Rc))
    return 3;
  if (pl->runs3 && interp_tc_supported(3, pl->s, rc)) return 2;
  return interp_tc_supported(3, pl->s, rc) ? 1 : 0;
}

// Stage timing: a pair of events around a group of launches on `st`.
struct StageTimer {
  agp_plan_s* pl;
  int stage, dim;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageTimer(agp_plan_s* p, int s, cudaStream_t t, int d = 0) : pl(p), stage(s), dim(d), st(t) {
    if (pl->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  ~StageTimer() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) == cudaSuccess && cudaEventRecord(b, st) == cudaSuccess)
      pl->prof_ev.push_back({stage, dim, a, b});
    else
      cudaEventDestroy(a);
  }
};

// Spectra of a block of right-hand sides, as agp_matvec_spectra stores them:
// the windows in the order of the plan's DFT groups (a group = the windows of
// one (d, N)), each window's Hermitian-half spectrum [K^(d-1) Kh] x R complex
// (plan precision), the forward DFT of the spread grid before deconvolution.
// k_save_spectra copies columns r0 .. r0 + Rc - 1 of one pass for every
// window of a group (blockIdx.y: the window within the group).
template <typename T2>
__global__ void k_save_spectra(const FftWin* __restrict__ tab, int sel, int64_t E, int rc, int Rc,
                               int R, int r0, T2* __restrict__ out) {
  const FftWin f = tab[blockIdx.y];
  const T2* spec = reinterpret_cast<const T2*>(sel == 1 ? f.specA : f.specB);
  T2* o = out + (int64_t)blockIdx.y * E * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E * Rc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / Rc;
    const int c = (int)(e - k * Rc);
    o[k * R + r0 + c] = spec[k * rc + c];
  }
}

// out[c] += scale sum_s sum_k w_k D_k Re(conj(A_k) B_k) over the windows of
// one group, D = the spectral multiplier of the kernel (der = 0) or of its
// ell-derivative (der = 1), w_k = 1 for k_d = 0 and 2 for k_d > 0 (the
// Hermitian half stands for the full symmetric index set). With A and B the
// spectra of G and V this is G^T (sum_s K_s) V (der = 0) or
// G^T (sum_s K_s^der) V (der = 1) for the operator agp_matvec applies:
// interpolation is the transpose of spreading. FP64 accumulation.
constexpr int kFormThreads = 256;
template <typename T, typename T2>
__global__ void __launch_bounds__(kFormThreads)
k_spec_form(const FftWin* __restrict__ tab, int der, const T2* __restrict__ A,
            const T2* __restrict__ B, int64_t E, int Kh, int R, double scale,
            double* __restrict__ out) {
  __shared__ double red[kFormThreads / 32][32];
  const FftWin f = tab[blockIdx.y];
  const T* dm = reinterpret_cast<const T*>(der ? f.dmul_der : f.dmul);
  const T2* a = A + (int64_t)blockIdx.y * E * R;
  const T2* b = B + (int64_t)blockIdx.y * E * R;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c = blockIdx.z * 32 + lane;
  double acc = 0.0;
  if (c < R)
    for (int64_t k = blockIdx.x * (int64_t)(kFormThreads / 32) + warp; k < E;
         k += (int64_t)gridDim.x * (kFormThreads / 32)) {
      const T2 x = a[k * R + c], y = b[k * R + c];
      const double w = (k % Kh == 0) ? 1.0 : 2.0;
      acc += w * (double)dm[k] * ((double)x.x * (double)y.x + (double)x.y * (double)y.y);
    }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < R) {
    double sum = 0.0;
    for (int q = 0; q < kFormThreads / 32; ++q) sum += red[q][lane];
    atomicAdd(out + c, scale * sum);
  }
}

// Sum over windows of scale * K_s V (coefficient set `der`), added into Out.
// With spec: the forward spectra of V are also stored there (layout of
// k_save_spectra); with spec_only, nothing else is done (Out unused).
template <typename T>
agp_status apply_windows(agp_plan_s* pl, const T* V, int64_t ldv, T* Out, int64_t ldo, int R,
                         int der, T scale, cudaStream_t st, void* spec = nullptr,
                         bool spec_only = false) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const WinDev<T>* wins = reinterpret_cast<const WinDev<T>*>(pl->wins_dev);
  for (int r0 = 0, rc = 0; r0 < R; r0 += rc) {
    rc = pick_rc(pl, R - r0);
    const int Rc = R - r0 < rc ? R - r0 : rc;
    {
      StageTimer tm(pl, 3, st);
      for (const auto& g : pl->groups) AGP_CUDA(zero_grids<T>(g, rc, st));
      pl->launches[3] += (int64_t)pl->groups.size();
    }
    // the d = 3 windows first on `st`; the others on the side stream next to
    // it when both are present (separate grids; forked and joined by events)
    const bool split = pl->items_by_d[3] > pl->items_by_d[2] &&
                       pl->items_by_d[2] > pl->items_by_d[0] && pl->side;
    if (split) {
      AGP_CUDA(cudaEventRecord(pl->fork_ev, st));
      AGP_CUDA(cudaStreamWaitEvent(pl->side, pl->fork_ev, 0));
    }
    for (int q = 0; q < kMaxDim; ++q) {
      const int dd = kMaxDim - q;
      const int64_t a = pl->items_by_d[dd - 1], b = pl->items_by_d[dd];
      if (b == a) continue;
      cudaStream_t sd = (split && dd < 3) ? pl->side : st;
      StageTimer tm(pl, 0, sd, dd);
      const int fam = dd == 3 ? spread_family3(pl, rc) : 0;
      if (fam == 3)
        AGP_CUDA(spread_units_tm(
            reinterpret_cast<const WinDev<float>*>(wins),
            static_cast<const unsigned char*>(pl->grid_maps) +
                (size_t)(rc == 32 ? pl->P : 0) * kGridMapBytes,
            pl->P, pl->runs3, pl->n_runs3, pl->s, reinterpret_cast<const float*>(V + r0), ldv, Rc,
            rc, pl->err_dev, pl->wait_limit, st));
      else if (fam == 2)
        AGP_CUDA(spread_items_sel<T>(wins, nullptr, pl->runs3, pl->n_runs3, dd, pl->s, rc, V + r0,
                                     ldv, Rc, 1, pl->err_dev, pl->wait_limit, st));
      else
        AGP_CUDA(spread_items_sel<T>(wins, nullptr, pl->items_all + a, b - a, dd, pl->s, rc,
                                     V + r0, ldv, Rc, pl->use_tc, pl->err_dev, pl->wait_limit,
                                     sd));
      pl->launches[0] += 1;
    }
    if (split) {
      AGP_CUDA(cudaEventRecord(pl->join_ev, pl->side));
      AGP_CUDA(cudaStreamWaitEvent(st, pl->join_ev, 0));
    }
    {
      StageTimer tm(pl, 1, st);
      // groups with d = 2 or 3 take the three-launch stage unless their
      // spectra are kept (at most 8 such groups: d in {2, 3} x 4 sizes N)
      FftGroup fg[8];
      int nf = 0;
      if (!spec)
        for (const auto& g : pl->groups)
          if (dft_fused_supported(g) && nf < 8) fg[nf++] = g;
      if (nf > 0) {
        AGP_CUDA(dft_stage<T>(fg, nf, der, rc, st));
        pl->launches[1] += 3;
      }
      int64_t goff = 0;
      for (const auto& g : pl->groups) {
        bool done = false;
        for (int q = 0; q < nf; ++q) done = done || fg[q].tab == g.tab;
        if (done) continue;
        AGP_CUDA(fft_forward<T>(g, rc, st));
        pl->launches[1] += g.d;
        if (spec) {
          const unsigned bx = (unsigned)std::min<int64_t>(nblk(g.dmul_elems * Rc, 256), 1024);
          k_save_spectra<T2><<<dim3(bx, g.count), 256, 0, st>>>(
              g.tab, (g.d % 2) ? 1 : 2, g.dmul_elems, rc, Rc, R, r0,
              reinterpret_cast<T2*>(spec) + goff);
          pl->launches[1] += 1;
          goff += (int64_t)g.count * g.dmul_elems * R;
        }
        if (spec_only) continue;
        AGP_CUDA(spectral_multiply<T>(g, der, rc, st));
        AGP_CUDA(fft_inverse<T>(g, rc, st));
        pl->launches[1] += g.d + 1;
      }
    }
    if (spec_only) continue;
    if (split) {
      AGP_CUDA(cudaEventRecord(pl->fork_ev, st));
      AGP_CUDA(cudaStreamWaitEvent(pl->side, pl->fork_ev, 0));
    }
    for (int q = 0; q < kMaxDim; ++q) {
      const int dd = kMaxDim - q;
      const int64_t a = pl->items_by_d[dd - 1], b = pl->items_by_d[dd];
      if (b == a) continue;
      cudaStream_t sd = (split && dd < 3) ? pl->side : st;
      StageTimer tm(pl, 2, sd, dd);
      const int fam = dd == 3 ? interp_family3(pl, rc, Rc) : 0;
      if (fam == 3)
        AGP_CUDA(interp_units_tm(reinterpret_cast<const WinDev<float>*>(wins), pl->P, pl->runs3,
                                 pl->n_runs3, pl->s, reinterpret_cast<float*>(Out + r0), ldo, Rc,
                                 (float)scale, rc, pl->err_dev, pl->wait_limit, st));
      else if (fam == 2)
        AGP_CUDA(interp_items_sel<T>(wins, nullptr, pl->runs3, pl->n_runs3, dd, pl->s, rc,
                                     Out + r0, ldo, Rc, scale, 1, pl->err_dev, pl->wait_limit,
                                     st));
      else
        AGP_CUDA(interp_items_sel<T>(wins, nullptr, pl->items_all + a, b - a, dd, pl->s, rc,
                                     Out + r0, ldo, Rc, scale, pl->use_tc, pl->err_dev,
                                     pl->wait_limit, sd));
      pl->launches[2] += 1;
    }
    if (split) {
      AGP_CUDA(cudaEventRecord(pl->join_ev, pl->side));
      AGP_CUDA(cudaStreamWaitEvent(st, pl->join_ev, 0));
    }
  }
  return AGP_OK;
}

template <typename T>
agp_status matvec_t(agp_plan_s* pl, const T* V, int64_t ldv, T* Out, int64_t ldo, int R,
                    T noise, T scale, int der, bool windows, cudaStream_t st,
                    void* spec = nullptr) {
  if (Out) {
    StageTimer tm(pl, 3, st);
    k_init_out<T><<<nblk(pl->n * R, 256), 256, 0, st>>>(Out, ldo, V, ldv, pl->n, R, noise);
    pl->launches[3] += 1;
  }
  AGP_CUDA(cudaGetLastError());
  if (windows) AGP_TRY(apply_windows<T>(pl, V, ldv, Out, ldo, R, der, scale, st, spec, !Out));
  return AGP_OK;
}

int64_t spectra_elems(const agp_plan_s* pl, int R) {
  int64_t e = 0;
  for (const auto& g : pl->groups) e += (int64_t)g.count * g.dmul_elems * R;
  return e;
}

template <typename T>
agp_status spectral_form_t(agp_plan_s* pl, int der, double scale, const void* A, const void* B,
                           int R, double* out, cudaStream_t st) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  AGP_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * R, st));
  int64_t goff = 0;
  for (const auto& g : pl->groups) {
    const unsigned bx = (unsigned)std::min<int64_t>((g.dmul_elems + 63) / 64, 256);
    k_spec_form<T, T2><<<dim3(bx, g.count, (R + 31) / 32), kFormThreads, 0, st>>>(
        g.tab, der, reinterpret_cast<const T2*>(A) + goff, reinterpret_cast<const T2*>(B) + goff,
        g.dmul_elems, g.N / 2 + 1, R, scale, out);
    pl->launches[1] += 1;
    goff += (int64_t)g.count * g.dmul_elems * R;
  }
  return cuda_status(cudaGetLastError(), "spectral_form");
}

agp_status check_block(agp_plan pl, const void* V, int64_t ldv, const void* Out, int64_t ldo,
                       int R) {
  if (!pl) return set_error(AGP_EINVAL, "plan is NULL");
  if (!V || !Out) return set_error(AGP_EINVAL, "V / Out is NULL");
  if (R < 1 || ldv < R || ldo < R) return set_error(AGP_EINVAL, "need R >= 1, ldv >= R, ldo >= R");
  const size_t es = elem_size(pl->prec);
  const char* v0 = static_cast<const char*>(V);
  const char* o0 = static_cast<const char*>(Out);
  const char* v1 = v0 + es * (size_t)((pl->n - 1) * ldv + R);
  const char* o1 = o0 + es * (size_t)((pl->n - 1) * ldo + R);
  if (v0 < o1 && o0 < v1) return set_error(AGP_EINVAL, "Out overlaps V");
  return AGP_OK;
}

template <typename T>
struct Cplx;
template <>
struct Cplx<float> { using t = float2; };
template <>
struct Cplx<double> { using t = double2; };

// Adjoint NFFT of one window: spread, forward DFT, deconvolve (Appendix A).
template <typename T>
agp_status adjoint_nfft_t(agp_plan_s* pl, int window, const T* V, int64_t ldv, int R, void* chat,
                          cudaStream_t st) {
  using T2 = typename Cplx<T>::t;
  Window& w = pl->win[window];
  const FftGroup g = w.self_group();
  const int rc = pick_rc(pl, R);
  const WinDev<T>* wins = reinterpret_cast<const WinDev<T>*>(pl->wins_dev);
  for (int r0 = 0; r0 < R; r0 += rc) {
    const int Rc = R - r0 < rc ? R - r0 : rc;
    AGP_CUDA(zero_grids<T>(g, rc, st));
    AGP_CUDA(spread_items_sel<T>(wins, nullptr, w.items, w.n_items, w.d, pl->s, rc, V + r0, ldv,
                                 Rc, pl->use_tc, pl->err_dev, pl->wait_limit, st));
    AGP_CUDA(fft_forward<T>(g, rc, st));
    const T2* spec = (const T2*)((w.d % 2) ? w.specA : w.specB);
    k_extract_spectrum<T, T2><<<nblk(w.cells * Rc, 256), 256, 0, st>>>(
        spec, (const double*)w.winhat, w.N, w.d, rc, Rc, (T2*)chat + (int64_t)r0 * w.cells);
    AGP_CUDA(cudaGetLastError());
  }
  return AGP_OK;
}

// Real part of the NFFT of one window: deconvolve, inverse DFT, interpolate.
template <typename T>
agp_status nfft_real_t(agp_plan_s* pl, int window, const void* fhat, int R, T* Out, int64_t ldo,
                       cudaStream_t st) {
  using T2 = typename Cplx<T>::t;
  Window& w = pl->win[window];
  const FftGroup g = w.self_group();
  const int rc = pick_rc(pl, R);
  const int64_t spec_total = w.dmul_elems * rc;
  const WinDev<T>* wins = reinterpret_cast<const WinDev<T>*>(pl->wins_dev);
  k_init_out<T><<<nblk(pl->n * R, 256), 256, 0, st>>>(Out, ldo, nullptr, 0, pl->n, R, T(0));
  for (int r0 = 0; r0 < R; r0 += rc) {
    const int Rc = R - r0 < rc ? R - r0 : rc;
    T2* spec = (T2*)((w.d % 2) ? w.specA : w.specB);
    k_insert_spectrum<T, T2><<<nblk(spec_total, 256), 256, 0, st>>>(
        (const T2*)fhat + (int64_t)r0 * w.cells, (const double*)w.winhat, w.N, w.d, rc, Rc, spec);
    AGP_CUDA(fft_inverse<T>(g, rc, st));
    AGP_CUDA(interp_items<T>(wins, nullptr, w.items, w.n_items, w.d, pl->s, rc, Out + r0, ldo, Rc,
                             T(1), st));
  }
  return cuda_status(cudaGetLastError(), "agp_nfft_real");
}

}  // namespace
}  // namespace agp

using namespace agp;

extern "C" {

const char* agp_status_string(agp_status s) {
  switch (s) {
    case AGP_OK: return "AGP_OK";
    case AGP_EINVAL: return "AGP_EINVAL";
    case AGP_EDOMAIN: return "AGP_EDOMAIN";
    case AGP_ECUDA: return "AGP_ECUDA";
    case AGP_ENOMEM: return "AGP_ENOMEM";
    case AGP_NOT_CONVERGED: return "AGP_NOT_CONVERGED";
    case AGP_TIMEOUT: return "AGP_TIMEOUT";
    case AGP_ENAN: return "AGP_ENAN";
  }
  return "AGP_UNKNOWN";
}

const char* agp_last_error(void) { return g_last_error.c_str(); }

agp_status agp_plan_create(agp_plan* out, const agp_plan_desc* d, void* stream) {
  if (!out) return set_error(AGP_EINVAL, "out is NULL");
  *out = nullptr;
  AGP_TRY(validate(d));
  auto* pl = new (std::nothrow) agp_plan_s();
  if (!pl) return set_error(AGP_ENOMEM, "host allocation");
  pl->n = d->n;
  pl->p = d->p;
  pl->P = d->P;
  pl->s = d->cutoff;
  pl->sigma_os = d->sigma_os;
  pl->kernel = d->kernel;
  pl->prec = d->prec;
  pl->ell = d->ell;
  pl->sigma_f = d->sigma_f;
  pl->sigma_eps = d->sigma_eps;
  pl->kb_b = M_PI * (2.0 - 1.0 / d->sigma_os);
  pl->kb_norm = 1.0 / (M_PI * bessel_i0(pl->kb_b * d->cutoff));
  pl->rc_max = d->prec == AGP_F32 ? 32 : 4;
  pl->win.resize(d->P);
  for (int s = 0; s < d->P; ++s) {
    Window& w = pl->win[s];
    w.d = d->win_ptr[s + 1] - d->win_ptr[s];
    for (int t = 0; t < w.d; ++t) w.feat[t] = d->win_feat[d->win_ptr[s] + t];
    w.N = d->N[s];
    w.n_os = d->sigma_os * w.N;
    w.s = d->cutoff;
    w.W = w.N + 2 * w.s - 1;
    w.K = w.N + 1;
    w.Kh = w.N / 2 + 1;
    w.cells = 1;
    w.grid_elems = 1;
    w.spec_elems = w.Kh;
    w.dmul_elems = w.Kh;
    for (int t = 0; t < w.d; ++t) {
      w.cells *= w.N;
      w.grid_elems *= w.W;
    }
    for (int t = 0; t < w.d - 1; ++t) {
      w.spec_elems *= w.W;
      w.dmul_elems *= w.K;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  agp_status s = (d->prec == AGP_F32) ? plan_build<float>(pl, d, st) : plan_build<double>(pl, d, st);
  if (s != AGP_OK) {
    cudaStreamSynchronize(st);
    free_plan(pl);
    return s;
  }
  *out = pl;
  return AGP_OK;
}

agp_status agp_plan_destroy(agp_plan pl) {
  if (!pl) return AGP_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(pl);
  return cuda_status(e, "agp_plan_destroy");
}

agp_status agp_set_hyper(agp_plan pl, double ell, double sigma_f, double sigma_eps, void* stream) {
  if (!pl) return set_error(AGP_EINVAL, "plan is NULL");
  if (!(ell > 0) || !std::isfinite(ell) || !std::isfinite(sigma_f) || !std::isfinite(sigma_eps))
    return set_error(AGP_EINVAL, "bad hyperparameters");
  const bool new_ell = ell != pl->ell;
  pl->ell = ell;
  pl->sigma_f = sigma_f;
  pl->sigma_eps = sigma_eps;
  if (!new_ell) return AGP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return pl->prec == AGP_F32 ? compute_coeffs<float>(pl, st) : compute_coeffs<double>(pl, st);
}

agp_status agp_matvec(agp_plan pl, const void* V, int64_t ldv, void* Out, int64_t ldo, int R,
                      int add_noise, void* stream) {
  AGP_TRY(check_block(pl, V, ldv, Out, ldo, R));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double noise = add_noise ? pl->sigma_eps * pl->sigma_eps : 0.0;
  const double scale = pl->sigma_f * pl->sigma_f;
  if (pl->prec == AGP_F32)
    return matvec_t<float>(pl, (const float*)V, ldv, (float*)Out, ldo, R, (float)noise,
                           (float)scale, 0, true, st);
  return matvec_t<double>(pl, (const double*)V, ldv, (double*)Out, ldo, R, noise, scale, 0, true,
                          st);
}

agp_status agp_spectra_size(agp_plan pl, int R, int64_t* elems) {
  if (!pl || R < 1 || !elems) return set_error(AGP_EINVAL, "bad arguments");
  *elems = spectra_elems(pl, R);
  return AGP_OK;
}

agp_status agp_matvec_spectra(agp_plan pl, const void* V, int64_t ldv, void* Out, int64_t ldo,
                              int R, int add_noise, void* spec, void* stream) {
  if (!pl || !spec) return set_error(AGP_EINVAL, "bad arguments");
  if (Out) {
    AGP_TRY(check_block(pl, V, ldv, Out, ldo, R));
  } else if (!V || R < 1 || ldv < R) {
    return set_error(AGP_EINVAL, "need V, R >= 1, ldv >= R");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double noise = add_noise ? pl->sigma_eps * pl->sigma_eps : 0.0;
  const double scale = pl->sigma_f * pl->sigma_f;
  if (pl->prec == AGP_F32)
    return matvec_t<float>(pl, (const float*)V, ldv, (float*)Out, ldo, R, (float)noise,
                           (float)scale, 0, true, st, spec);
  return matvec_t<double>(pl, (const double*)V, ldv, (double*)Out, ldo, R, noise, scale, 0, true,
                          st, spec);
}

agp_status agp_spectral_form(agp_plan pl, int which, const void* A, const void* B, int R,
                             double* out, void* stream) {
  if (!pl || !A || !B || !out || R < 1) return set_error(AGP_EINVAL, "bad arguments");
  double scale = 0.0;
  int der = 0;
  switch (which) {
    case -1: scale = pl->sigma_f * pl->sigma_f; break;
    case AGP_D_ELL: scale = pl->sigma_f * pl->sigma_f; der = 1; break;
    case AGP_D_SIGMA_F: scale = 2.0 * pl->sigma_f; break;
    default: return set_error(AGP_EINVAL, "which must be -1, AGP_D_ELL or AGP_D_SIGMA_F");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl->prec == AGP_F32) return spectral_form_t<float>(pl, der, scale, A, B, R, out, st);
  return spectral_form_t<double>(pl, der, scale, A, B, R, out, st);
}

agp_status agp_deriv_matvec(agp_plan pl, agp_param which, const void* V, int64_t ldv, void* Out,
                            int64_t ldo, int R, void* stream) {
  AGP_TRY(check_block(pl, V, ldv, Out, ldo, R));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double noise = 0.0, scale = 0.0;
  int der = 0;
  bool windows = true;
  switch (which) {
    case AGP_D_ELL: scale = pl->sigma_f * pl->sigma_f; der = 1; break;
    case AGP_D_SIGMA_F: scale = 2.0 * pl->sigma_f; break;
    case AGP_D_SIGMA_EPS: noise = 2.0 * pl->sigma_eps; windows = false; break;
    default: return set_error(AGP_EINVAL, "bad agp_param");
  }
  if (pl->prec == AGP_F32)
    return matvec_t<float>(pl, (const float*)V, ldv, (float*)Out, ldo, R, (float)noise,
                           (float)scale, der, windows, st);
  return matvec_t<double>(pl, (const double*)V, ldv, (double*)Out, ldo, R, noise, scale, der,
                          windows, st);
}

agp_status agp_adjoint_nfft(agp_plan pl, int window, const void* V, int64_t ldv, int R, void* chat,
                            void* stream) {
  if (!pl || window < 0 || window >= pl->P || !V || !chat || R < 1 || ldv < R)
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl->prec == AGP_F32)
    return adjoint_nfft_t<float>(pl, window, (const float*)V, ldv, R, chat, st);
  return adjoint_nfft_t<double>(pl, window, (const double*)V, ldv, R, chat, st);
}

agp_status agp_nfft_real(agp_plan pl, int window, const void* fhat, int R, void* Out, int64_t ldo,
                         void* stream) {
  if (!pl || window < 0 || window >= pl->P || !fhat || !Out || R < 1 || ldo < R)
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl->prec == AGP_F32) return nfft_real_t<float>(pl, window, fhat, R, (float*)Out, ldo, st);
  return nfft_real_t<double>(pl, window, fhat, R, (double*)Out, ldo, st);
}

agp_status agp_plan_bins(agp_plan pl, int window, int32_t* bins, void* stream) {
  if (!pl || window < 0 || window >= pl->P || !bins) return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Window& w = pl->win[window];
  if (pl->prec == AGP_F32)
    k_bins_out<float><<<nblk(pl->n, 256), 256, 0, st>>>((const float*)w.xs, w.perm, pl->n, w.d,
                                                        w.n_os, bins);
  else
    k_bins_out<double><<<nblk(pl->n, 256), 256, 0, st>>>((const double*)w.xs, w.perm, pl->n, w.d,
                                                         w.n_os, bins);
  return cuda_status(cudaGetLastError(), "agp_plan_bins");
}

agp_status agp_plan_coeffs(agp_plan pl, int window, int deriv, double* b, void* stream) {
  if (!pl || window < 0 || window >= pl->P || !b) return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Window& w = pl->win[window];
  AGP_CUDA(cudaMemcpyAsync(b, deriv ? w.bder : w.b, sizeof(double) * w.cells,
                           cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  return AGP_OK;
}

agp_status agp_profile_enable(agp_plan pl, int enable) {
  if (!pl) return set_error(AGP_EINVAL, "plan is NULL");
  pl->prof = enable != 0;
  return AGP_OK;
}

agp_status agp_profile_read(agp_plan pl, agp_profile_t* out, int reset, void* stream) {
  if (!pl || !out) return set_error(AGP_EINVAL, "bad arguments");
  AGP_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  for (int k = 0; k < 4; ++k) {
    out->ms[k] = 0.0;
    out->launches[k] = pl->launches[k];
    for (int d = 0; d < 4; ++d) {
      out->ms_by_dim[k][d] = 0.0;
      out->timed_by_dim[k][d] = 0;
    }
  }
  for (auto& e : pl->prof_ev) {
    float ms = 0.f;
    AGP_CUDA(cudaEventSynchronize(e.b));
    AGP_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
    out->ms[e.stage] += ms;
    out->ms_by_dim[e.stage][e.dim] += ms;
    out->timed_by_dim[e.stage][e.dim] += 1;
  }
  if (reset) {
    for (auto& e : pl->prof_ev) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    pl->prof_ev.clear();
    for (int k = 0; k < 4; ++k) pl->launches[k] = 0;
  }
  return AGP_OK;
}

agp_status agp_plan_set_tensor_cores(agp_plan pl, int enable) {
  if (!pl || enable < 0 || enable > 3) return set_error(AGP_EINVAL, "bad arguments");
  pl->use_tc = enable;
  return AGP_OK;
}

agp_status agp_plan_set_boundary(agp_plan pl, double eps_b, int p, void* stream) {
  if (!pl) return set_error(AGP_EINVAL, "plan is NULL");
  if (!(eps_b >= 0.0) || !(eps_b <= 0.25) || p < 0 || p > kBndMaxP)
    return set_error(AGP_EINVAL, "boundary smoothing needs 0 <= eps_b <= 1/4 and 0 <= p <= 8");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool on = eps_b > 0.0 && p > 0;
  if (on) {
    // every window's points inside the ball |x| <= 1/4 - eps_b/2, so that all
    // differences have |x_i - x_j| <= 1/2 - eps_b, where kappa_R = kappa
    unsigned long long* mx = nullptr;
    AGP_CUDA(cudaMallocAsync(&mx, sizeof(unsigned long long) * pl->P, st));
    AGP_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * pl->P, st));
    for (int w = 0; w < pl->P; ++w) {
      const Window& win = pl->win[w];
      const int blocks = (int)std::min<int64_t>(nblk(pl->n, 256), 1216);
      if (pl->prec == AGP_F32)
        k_max_norm2<float><<<blocks, 256, 0, st>>>(reinterpret_cast<const float*>(win.xs), pl->n,
                                                   win.d, mx + w);
      else
        k_max_norm2<double><<<blocks, 256, 0, st>>>(reinterpret_cast<const double*>(win.xs),
                                                    pl->n, win.d, mx + w);
    }
    AGP_CUDA(cudaGetLastError());
    std::vector<unsigned long long> h(pl->P);
    AGP_CUDA(cudaMemcpyAsync(h.data(), mx, sizeof(unsigned long long) * pl->P,
                             cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaFreeAsync(mx, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    const double rad = 0.25 - 0.5 * eps_b;
    for (int w = 0; w < pl->P; ++w) {
      double r2;
      std::memcpy(&r2, &h[w], sizeof r2);
      if (!(r2 <= rad * rad))
        return set_error(AGP_EDOMAIN, "boundary smoothing needs every window's points in the "
                                      "ball |x| <= 1/4 - eps_b/2");
    }
    if (!pl->bnd_poly) AGP_CUDA(cudaMalloc(&pl->bnd_poly, sizeof(double) * 2 * kBndStride));
  }
  pl->bnd_eps = on ? eps_b : 0.0;
  pl->bnd_p = on ? p : 0;
  return pl->prec == AGP_F32 ? compute_coeffs<float>(pl, st) : compute_coeffs<double>(pl, st);
}

agp_status agp_plan_set_wait_limit(agp_plan pl, int64_t polls) {
  if (!pl || polls < 0) return set_error(AGP_EINVAL, "bad arguments");
  pl->wait_limit = polls == 0 ? kDefaultWaitLimit : (long long)polls;
  return AGP_OK;
}

agp_status agp_plan_check(agp_plan pl, void* stream) {
  if (!pl) return set_error(AGP_EINVAL, "bad arguments");
  return timeout_check(pl, static_cast<cudaStream_t>(stream));
}

agp_status agp_plan_set_item_points(agp_plan pl, int points, void* stream) {
  if (!pl || points < 16 || points > 4096)
    return set_error(AGP_EINVAL, "points per work item must be in [16, 4096]");
  return build_items(pl, points, static_cast<cudaStream_t>(stream));
}

agp_status agp_plan_autotune(agp_plan pl, int R, int reps, int* points, double* ms, void* stream) {
  if (!pl || R < 1 || reps < 1) return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // cache key: precision, cutoff, pass width, (d, N) of every window, log2 n
  std::string key = std::to_string((int)pl->prec) + "/" + std::to_string(pl->s) + "/" +
                    std::to_string(pick_rc(pl, R)) + "/" + std::to_string(std::min(R, 32)) + "/";
  for (const auto& w : pl->win) key += std::to_string(w.d) + "x" + std::to_string(w.N) + ",";
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= pl->n) ++lg;
  key += "/" + std::to_string(lg);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tune_cache.find(key);
    if (f != g_tune_cache.end()) {
      pl->use_tc = f->second.mode;
      AGP_TRY(build_items(pl, f->second.points, st));
      if (points) *points = f->second.points;
      if (ms) *ms = f->second.ms;
      return AGP_OK;
    }
  }
  const size_t bytes = (size_t)pl->n * R * (pl->prec == AGP_F32 ? 4 : 8);
  void *V = nullptr, *Out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  struct Free {
    void **v, **o;
    cudaEvent_t *a, *b;
    cudaStream_t st;
    ~Free() {
      if (*v) cudaFreeAsync(*v, st);
      if (*o) cudaFreeAsync(*o, st);
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } fr{&V, &Out, &a, &b, st};
  AGP_CUDA(cudaMallocAsync(&V, bytes, st));
  AGP_CUDA(cudaMallocAsync(&Out, bytes, st));
  AGP_CUDA(cudaMemsetAsync(V, 0, bytes, st));
  AGP_CUDA(cudaEventCreate(&a));
  AGP_CUDA(cudaEventCreate(&b));
  auto time_it = [&](float* t) -> agp_status {
    AGP_TRY(agp_matvec(pl, V, R, Out, R, R, 1, st));   // warm-up
    AGP_CUDA(cudaEventRecord(a, st));
    for (int k = 0; k < reps; ++k) AGP_TRY(agp_matvec(pl, V, R, Out, R, R, 1, st));
    AGP_CUDA(cudaEventRecord(b, st));
    AGP_CUDA(cudaEventSynchronize(b));
    AGP_CUDA(cudaEventElapsedTime(t, a, b));
    *t /= reps;
    return AGP_OK;
  };
  // stage 1: the kernel family (tensor-core pairings or FMA pipes; FP32
  // plans only) at the current work-item size; stage 2: the work-item size
  int best_mode = pl->use_tc, best_pts = pl->item_points;
  float best_ms = 0.0f;
  const int modes[] = {1, 2, 3, 0};
  for (int md : modes) {
    if (pl->prec != AGP_F32 && md != 0) continue;
    pl->use_tc = md;
    float t = 0.0f;
    AGP_TRY(time_it(&t));
    if (best_ms == 0.0f || t < best_ms) {
      best_ms = t;
      best_mode = md;
    }
  }
  pl->use_tc = best_mode;
  const int cands[] = {64, 128, 256, 512, 1024};
  for (int c : cands) {
    AGP_TRY(build_items(pl, c, st));
    float t = 0.0f;
    AGP_TRY(time_it(&t));
    if (t < best_ms) {
      best_ms = t;
      best_pts = c;
    }
  }
  AGP_TRY(build_items(pl, best_pts, st));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = TuneEntry{best_mode, best_pts, (double)best_ms};
  }
  if (points) *points = best_pts;
  if (ms) *ms = best_ms;
  return AGP_OK;
}

agp_status agp_plan_tensor_cores(agp_plan pl, int* mode) {
  if (!pl || !mode) return set_error(AGP_EINVAL, "bad arguments");
  *mode = pl->use_tc;
  return AGP_OK;
}

agp_status agp_plan_kernel_families(agp_plan pl, int R, int64_t ldv, int* spread, int* interp) {
  if (!pl || R < 1 || ldv < R || !spread || !interp) return set_error(AGP_EINVAL, "bad arguments");
  *spread = *interp = -1;
  bool d3 = false;
  for (const Window& w : pl->win) d3 = d3 || w.d == 3;
  if (!d3) return AGP_OK;
  const int rc = pick_rc(pl, R);
  *spread = spread_family3(pl, rc);
  *interp = interp_family3(pl, rc, std::min(rc, R));
  return AGP_OK;
}

agp_status agp_autotune_clear_cache(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  return AGP_OK;
}

agp_status agp_plan_query(agp_plan pl, int64_t* n, int* P, int window, int* d, int* N,
                          int64_t* n_items) {
  if (!pl) return set_error(AGP_EINVAL, "plan is NULL");
  if (n) *n = pl->n;
  if (P) *P = pl->P;
  if (window >= 0 && window < pl->P) {
    if (d) *d = pl->win[window].d;
    if (N) *N = pl->win[window].N;
    if (n_items) *n_items = pl->win[window].n_items;
  }
  return AGP_OK;
}

}  // extern "C"
