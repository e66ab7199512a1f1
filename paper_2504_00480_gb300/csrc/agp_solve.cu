// Batched conjugate gradients, stochastic Lanczos quadrature and the
// negative log marginal likelihood gradient (Sec. 1 eqs. (1.2), (1.4), (1.5)
// with M = I).
//
// Blocks are RHS-minor [n][R]. The kernel matvecs run in the plan precision
// (FP32 or FP64); the CG recursion vectors x, r, p and every scalar (column
// dot products, alpha, beta, residual norms, the Lanczos matrix, its
// eigenvalues and the log determinant) are FP64 on the device. Column dot
// products are two-pass and deterministic: per-block partial sums in FP64,
// then one ordered sum per column. The host loop enqueues one CG iteration at
// a time and reads the per-column convergence flags back every few iterations.
#include <cmath>
#include <mutex>
#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

constexpr int kDotThreads = 256;   // 8 row groups x 32 columns
constexpr int kDotRows = 8;
constexpr int kMaxDotBlocks = 1024;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// partial[b][c] = sum over this block's rows of A[i][c] * B[i][c] (FP64), for
// the 32 columns c0 .. c0+31 of blockIdx.y.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kDotThreads)
k_dot_partial(const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B, int64_t ldb, int64_t n,
              int R, double* __restrict__ partial) {
  __shared__ double red[kDotRows][32];
  const int lane = threadIdx.x % 32, grp = threadIdx.x / 32;
  const int c = blockIdx.y * 32 + lane;
  double acc = 0.0;
  if (c < R) {
    // four rows per trip with independent partial sums, so that four loads
    // of each operand are in flight per thread
    const int64_t step = (int64_t)gridDim.x * kDotRows;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t i = (int64_t)blockIdx.x * kDotRows + grp;
    for (; i + 3 * step < n; i += 4 * step) {
      acc += (double)A[i * lda + c] * (double)B[i * ldb + c];
      a1 += (double)A[(i + step) * lda + c] * (double)B[(i + step) * ldb + c];
      a2 += (double)A[(i + 2 * step) * lda + c] * (double)B[(i + 2 * step) * ldb + c];
      a3 += (double)A[(i + 3 * step) * lda + c] * (double)B[(i + 3 * step) * ldb + c];
    }
    for (; i < n; i += step) acc += (double)A[i * lda + c] * (double)B[i * ldb + c];
    acc = (acc + a1) + (a2 + a3);
  }
  red[grp][lane] = acc;
  __syncthreads();
  if (grp == 0 && c < R) {
    double s = 0.0;
    for (int g = 0; g < kDotRows; ++g) s += red[g][lane];
    partial[(int64_t)blockIdx.x * R + c] = s;
  }
}

// out[c] = sum_b partial[b][c]: one CTA per column, each thread a strided
// share of the blocks, then a fixed-order tree in shared memory (the same
// summation order on every call)
constexpr int kDotFinalThreads = 256;
__global__ void __launch_bounds__(kDotFinalThreads)
k_dot_final(const double* __restrict__ partial, int nb, int R, double* __restrict__ out) {
  __shared__ double red[kDotFinalThreads];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kDotFinalThreads) s += partial[(int64_t)b * R + c];
  red[threadIdx.x] = s;
  __syncthreads();
#pragma unroll
  for (int h = kDotFinalThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

template <typename TS, typename TD>
__global__ void k_copy_block(const TS* __restrict__ src, int64_t lds, TD* __restrict__ dst,
                             int64_t ldd, int64_t n, int R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t i = e / R;
  const int c = (int)(e - i * R);
  dst[i * ldd + c] = (TD)src[i * lds + c];
}

template <typename T>
__global__ void k_zero_block(T* __restrict__ dst, int64_t ldd, int64_t n, int R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t i = e / R;
  dst[i * ldd + (e - i * R)] = T(0);
}

// Per-column CG state (FP64).
struct CgState {
  double* rr;       // current |r|^2
  double* bn2;      // |b|^2
  double* pq;       // p^T K p
  double* alpha;
  double* beta;
  double* relres;
  int* active;      // 1 while the column iterates
  int* iters;
  int* maxit;       // per-column iteration cap
  double* tol;      // per-column relative residual tolerance (0: run to maxit)
  double* ahist;    // [maxit_all][R]
  double* bhist;
  double* rz;       // r^T M^{-1} r (preconditioned runs)
  double* rznew;
  int pc;           // 1: preconditioned recursion
  // residual replacement (reliable updates; null when off)
  double* rr_ref;   // |r|^2 when r was last recomputed as b - K x
  int* want;        // 1: recompute r of this column at the next check
  int* fresh;       // 1: r of this column was recomputed in this iteration
};

__global__ void k_cg_start(CgState s, int R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  s.bn2[c] = s.rr[c];
  s.iters[c] = 0;
  s.relres[c] = s.rr[c] > 0.0 ? 1.0 : 0.0;
  s.active[c] = (s.rr[c] > 0.0 && s.maxit[c] > 0) ? 1 : 0;
  if (s.rr_ref) {
    s.rr_ref[c] = s.rr[c];
    s.want[c] = 0;
    s.fresh[c] = 0;
  }
}

// Residual replacement (reliable updates, after Sleijpen and van der Vorst):
// the recursion r_k = r_{k-1} - alpha K p drifts from b - K x_k when the
// operator carries rounding errors (FP32 plans; atomic accumulation makes
// them differ between applications). A column asks for its residual to be
// recomputed as b - K x once |r| has fallen 10x since the last
// recomputation, and before it may stop at the tolerance.
constexpr double kReplaceDrop2 = 1e-2;     // |r|^2 ratio that asks for a recomputation
constexpr double kReplaceJoin2 = 1e-1;     // ... and that joins one already asked for
__global__ void k_cg_want(CgState s, const double* __restrict__ rr_new, int R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  const double rn = rr_new[c];
  const bool conv = sqrt(rn / s.bn2[c]) <= s.tol[c];
  s.want[c] = s.active[c] && (rn < kReplaceDrop2 * s.rr_ref[c] || conv) ? 1
              : (s.active[c] && rn < kReplaceJoin2 * s.rr_ref[c] ? 2 : 0);
}

// x in the plan precision as x_hi + x_lo: part 0 writes x_hi = x rounded,
// part 1 x_lo = x - x_hi rounded (for FP64 plans x_lo = 0)
template <typename T>
__global__ void k_cg_xsplit(const double* __restrict__ x, T* __restrict__ xt, int part,
                            int64_t m) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m) return;
  const T hi = (T)x[e];
  xt[e] = part == 0 ? hi : (T)(x[e] - (double)hi);
}

// the columns being recomputed: r = b - q (part 0, q = K x_hi), then
// r -= q (part 1, q = K x_lo), so that r = b - K x without x's rounding to
// the plan precision
template <typename T>
__global__ void k_cg_replace(double* __restrict__ r, const T* __restrict__ B, int64_t ldb,
                             const T* __restrict__ q, const int* __restrict__ sel, int part,
                             int64_t n, int R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t i = e / R;
  const int c = (int)(e - i * R);
  if (!sel[c]) return;
  r[e] = (part == 0 ? (double)B[i * ldb + c] : r[e]) - (double)q[e];
}

__global__ void k_cg_replaced(CgState s, const double* __restrict__ rr_new, int R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  if (s.want[c]) {
    s.rr_ref[c] = rr_new[c];
    s.fresh[c] = 1;
  }
  s.want[c] = 0;
}

__global__ void k_cg_alpha(CgState s, int R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  // The truncated Fourier series of a kernel need not be positive definite
  // (no boundary smoothing), so p^T K p < 0 is possible and CG carries on as
  // the textbook recursion does; only an exact zero or a non-finite value
  // stops the column.
  double a = 0.0;
  if (s.active[c]) {
    const double pq = s.pq[c];
    if (pq != 0.0 && isfinite(pq)) {
      a = (s.pc ? s.rz[c] : s.rr[c]) / pq;
    } else {
      s.active[c] = 0;
    }
  }
  s.alpha[c] = a;
}

// x += alpha p, r -= alpha q (x, r, p FP64; q = K p in the plan precision)
template <typename T>
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                        const T* __restrict__ q, const double* __restrict__ alpha, int64_t n,
                        int R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int c = (int)(e % R);
  const double a = alpha[c];
  if (a == 0.0) return;
  x[e] += a * p[e];
  r[e] -= a * (double)q[e];
}

__global__ void k_cg_beta(CgState s, const double* __restrict__ rr_new, int it, int R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  double b = 0.0;
  if (s.active[c]) {
    const double rn = rr_new[c];
    if (s.pc) {
      b = s.rznew[c] / s.rz[c];
      s.rz[c] = s.rznew[c];
    } else {
      b = rn / s.rr[c];
    }
    s.ahist[(int64_t)it * R + c] = s.alpha[c];
    s.bhist[(int64_t)it * R + c] = b;
    s.iters[c] = it + 1;
    s.relres[c] = sqrt(rn / s.bn2[c]);
    s.rr[c] = rn;
    // with residual replacement a column stops at the tolerance only on a
    // recomputed residual
    const bool conv = s.relres[c] <= s.tol[c] && (!s.fresh || s.fresh[c]);
    if (!(rn > 0.0) || conv || it + 1 >= s.maxit[c]) s.active[c] = 0;
  }
  s.beta[c] = s.active[c] ? b : 0.0;
  if (s.fresh) s.fresh[c] = 0;
}

// p = r + beta p (FP64), and its copy in the plan precision for the next matvec
template <typename T>
__global__ void k_cg_p(double* __restrict__ p, T* __restrict__ pt, const double* __restrict__ r,
                       const double* __restrict__ beta, const int* __restrict__ active, int64_t n,
                       int R) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int c = (int)(e % R);
  if (!active[c]) return;
  const double v = r[e] + beta[c] * p[e];
  p[e] = v;
  pt[e] = (T)v;
}

// Lanczos matrix from the CG coefficients of one probe (the CG-Lanczos
// relation T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
// T_{j,j+1} = sqrt(beta_j)/alpha_j), its eigen-decomposition by the implicit
// QL method with Wilkinson shifts, and the Gauss quadrature
// z^T logm(K) z ~= |z|^2 sum_k tau_k^2 log theta_k, tau = first components of
// the eigenvectors (only the first row of the rotation product is kept).
constexpr int kMaxLanczos = 64;
constexpr int kSlqThreads = 32;

__device__ bool tridiag_ql(double* d, double* e, double* z, int m) {
  // d: diagonal; e[i] couples i and i+1 (e[m-1] = 0); z: first row of the
  // accumulated eigenvector matrix (starts as e_0).
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    while (true) {
      int mm = l;
      for (; mm < m - 1; ++mm)
        if (fabs(e[mm]) <= 1e-16 * (fabs(d[mm]) + fabs(d[mm + 1]))) break;
      if (mm == l) break;                       // d[l] has converged
      if (++iter > 60) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool split = false;
      for (int i = mm - 1; i >= l; --i) {
        double f = s * e[i];
        const double b = c * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {                         // the matrix splits at i+1
          d[i + 1] -= p;
          e[mm] = 0.0;
          split = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        f = z[i + 1];
        z[i + 1] = s * z[i] + c * f;
        z[i] = c * z[i] - s * f;
      }
      if (split) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  return true;
}

__global__ void __launch_bounds__(kSlqThreads)
k_slq_logdet(const double* __restrict__ ahist, const double* __restrict__ bhist,
             const int* __restrict__ iters, const double* __restrict__ bn2, int R, int c0,
             double* __restrict__ quad) {
  __shared__ double sd[kSlqThreads][kMaxLanczos];
  __shared__ double se[kSlqThreads][kMaxLanczos];
  __shared__ double sz[kSlqThreads][kMaxLanczos];
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  double* d = sd[threadIdx.x];
  double* e = se[threadIdx.x];
  double* z = sz[threadIdx.x];
  const int m = min(iters[c], kMaxLanczos);
  for (int j = 0; j < m; ++j) {
    const double aj = ahist[(int64_t)j * R + c];
    d[j] = 1.0 / aj + (j > 0 ? bhist[(int64_t)(j - 1) * R + c] / ahist[(int64_t)(j - 1) * R + c] : 0.0);
    e[j] = (j + 1 < m) ? sqrt(bhist[(int64_t)j * R + c]) / aj : 0.0;
    z[j] = (j == 0) ? 1.0 : 0.0;
  }
  if (m == 0 || !tridiag_ql(d, e, z, m)) {
    quad[c] = (m == 0) ? 0.0 : nan("");
    return;
  }
  double s = 0.0;
  for (int k = 0; k < m; ++k) s += z[k] * z[k] * log(d[k]);
  quad[c] = bn2[c] * s;
}

// CG workspace: the recursion vectors x, r, p are FP64 whatever the plan
// precision (the paper runs CG in double precision); the matvec reads pt, the
// copy of p in the plan precision, and writes q in the plan precision.
template <typename T>
struct Workspace {
  double *x = nullptr, *r = nullptr, *p = nullptr, *z = nullptr;
  T *pt = nullptr, *q = nullptr;
  double* partial = nullptr;
  double* scal = nullptr;   // 11 x R doubles
  int* iscal = nullptr;     // 3 x R ints
  double *ahist = nullptr, *bhist = nullptr;
  double* rz0 = nullptr;    // preconditioned runs: r_0^T M^{-1} r_0 per column
  cudaStream_t st;
  ~Workspace() {
    void* bufs[] = {x, z, r, p, pt, q, partial, scal, iscal, ahist, bhist, rz0};
    for (void* b : bufs)
      if (b) cudaFreeAsync(b, st);
  }
};

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

// ---- Column dot products without allocation (agp_dot_columns_static) --------
// The per-block FP64 partial sums of the two-pass reduction live in this
// file-scope device array instead of memory allocated per call: at most
// kStaticDotBlocks blocks x kStaticDotMaxR columns (256 KB). Every GPU that
// loads the library holds it until the process exits. Host code must not use
// the symbol as an address: static_dot_scratch() looks up its device address
// once per device (with that device current) and caches it.
constexpr int kStaticDotBlocks = 512;
constexpr int kStaticDotMaxR = 64;
constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_static_dot_scratch[kStaticDotBlocks * kStaticDotMaxR];

std::mutex g_static_dot_mu;
double* g_static_dot_addr[kMaxDevices] = {};

agp_status static_dot_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(AGP_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_dot_mu);
  if (!g_static_dot_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_dot_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
    g_static_dot_addr[dev] = static_cast<double*>(p);
  }
  *out = g_static_dot_addr[dev];
  return AGP_OK;
}

template <typename TA, typename TB>
agp_status col_dot(const TA* A, int64_t lda, const TB* B, int64_t ldb, int64_t n, int R,
                   double* partial, double* out, cudaStream_t st, agp_plan_s* pl) {
  const int nb = (int)std::min<int64_t>(kMaxDotBlocks, (n + kDotRows - 1) / kDotRows);
  dim3 grid(nb, (R + 31) / 32);
  k_dot_partial<TA, TB><<<grid, kDotThreads, 0, st>>>(A, lda, B, ldb, n, R, partial);
  k_dot_final<<<R, kDotFinalThreads, 0, st>>>(partial, nb, R, out);
  pl->launches[3] += 2;
  return cuda_status(cudaGetLastError(), "col_dot");
}

// CG on the columns of B; X receives the iterates. Per-column caps and
// tolerances come from maxit_h / tol_h. On return ws holds the alpha/beta
// history and the per-column state (scal layout: rr, bn2, pq, alpha, beta,
// relres, rrnew, spare; iscal: active, iters, maxit).
// With pc != nullptr (landmark preconditioner) or afn != nullptr (AFN) the
// recursion is preconditioned CG: z = M^{-1} r,
// alpha = r^T z / p^T K p, beta = r_new^T z_new / r^T z, p = z + beta p; the
// stopping test stays on the unpreconditioned relative residual.
// Batched (P)CG. With `reliable`, residual replacement (k_cg_want): at every
// check (each check_every iterations, check_every > 0) the columns that ask
// for it get r = b - K x, with x rounded to the plan precision for the
// matvec; a column stops at the tolerance only right after such a
// recomputation.
template <typename T>
agp_status cg_run(agp_plan_s* pl, const T* B, int64_t ldb, T* X, int64_t ldx, int R,
                  const std::vector<int>& maxit_h, const std::vector<double>& tol_h, int check_every,
                  Workspace<T>& ws, cudaStream_t st, const Precond* pc = nullptr,
                  const Afn* afn = nullptr, bool reliable = false) {
  const int64_t n = pl->n;
  const bool pcon = pc || afn;
  auto apply_pc = [&]() -> agp_status {
    pl->launches[3] += 1;
    return afn ? afn_apply(*afn, ws.r, R, ws.z, R, R, st) : precond_apply<T>(*pc, ws.r, ws.z, R, st);
  };
  int maxall = 0;
  for (int v : maxit_h) maxall = std::max(maxall, v);
  ws.st = st;
  AGP_CUDA(cudaMallocAsync(&ws.x, sizeof(double) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.r, sizeof(double) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.p, sizeof(double) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.pt, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.q, sizeof(T) * n * R, st));
  if (pcon) AGP_CUDA(cudaMallocAsync(&ws.z, sizeof(double) * n * R, st));
  if (pcon) AGP_CUDA(cudaMallocAsync(&ws.rz0, sizeof(double) * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.partial, sizeof(double) * kMaxDotBlocks * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.scal, sizeof(double) * 12 * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.iscal, sizeof(int) * 5 * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.ahist, sizeof(double) * std::max(1, maxall) * R, st));
  AGP_CUDA(cudaMallocAsync(&ws.bhist, sizeof(double) * std::max(1, maxall) * R, st));
  CgState s;
  s.rr = ws.scal;
  s.bn2 = ws.scal + R;
  s.pq = ws.scal + 2 * R;
  s.alpha = ws.scal + 3 * R;
  s.beta = ws.scal + 4 * R;
  s.relres = ws.scal + 5 * R;
  double* rrnew = ws.scal + 6 * R;
  s.tol = ws.scal + 7 * R;
  s.active = ws.iscal;
  s.iters = ws.iscal + R;
  s.maxit = ws.iscal + 2 * R;
  s.ahist = ws.ahist;
  s.bhist = ws.bhist;
  s.rz = ws.scal + 9 * R;
  s.rznew = ws.scal + 10 * R;
  s.pc = pcon ? 1 : 0;
  reliable = reliable && check_every > 0;
  s.rr_ref = reliable ? ws.scal + 11 * R : nullptr;
  s.want = reliable ? ws.iscal + 3 * R : nullptr;
  s.fresh = reliable ? ws.iscal + 4 * R : nullptr;
  AGP_CUDA(cudaMemcpyAsync(s.maxit, maxit_h.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMemcpyAsync(s.tol, tol_h.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));

  const unsigned gb = nblk(n * R, 256), gc = nblk(R, 128);
  k_zero_block<double><<<gb, 256, 0, st>>>(ws.x, R, n, R);
  k_copy_block<T, double><<<gb, 256, 0, st>>>(B, ldb, ws.r, R, n, R);
  pl->launches[3] += 2;
  if (pcon) {   // p = z = M^{-1} r, rz = r^T z
    AGP_TRY(apply_pc());
    k_copy_block<double, double><<<gb, 256, 0, st>>>(ws.z, R, ws.p, R, n, R);
    k_copy_block<double, T><<<gb, 256, 0, st>>>(ws.z, R, ws.pt, R, n, R);
    AGP_TRY(col_dot(ws.r, R, ws.z, R, n, R, ws.partial, s.rz, st, pl));
    AGP_CUDA(cudaMemcpyAsync(ws.rz0, s.rz, sizeof(double) * R, cudaMemcpyDeviceToDevice, st));
  } else {
    k_copy_block<T, double><<<gb, 256, 0, st>>>(B, ldb, ws.p, R, n, R);
    k_copy_block<T, T><<<gb, 256, 0, st>>>(B, ldb, ws.pt, R, n, R);
  }
  pl->launches[3] += 2;
  AGP_TRY(col_dot(ws.r, R, ws.r, R, n, R, ws.partial, s.rr, st, pl));
  k_cg_start<<<gc, 128, 0, st>>>(s, R);
  pl->launches[3] += 1;
  std::vector<int> act(R), want(R);
  for (int it = 0; it < maxall; ++it) {
    AGP_TRY(agp_matvec(pl, ws.pt, R, ws.q, R, R, 1, st));
    AGP_TRY(col_dot(ws.p, R, ws.q, R, n, R, ws.partial, s.pq, st, pl));
    k_cg_alpha<<<gc, 128, 0, st>>>(s, R);
    k_cg_xr<T><<<gb, 256, 0, st>>>(ws.x, ws.r, ws.p, ws.q, s.alpha, n, R);
    pl->launches[3] += 2;
    AGP_TRY(col_dot(ws.r, R, ws.r, R, n, R, ws.partial, rrnew, st, pl));
    if (reliable && (it + 1) % check_every == 0) {
      k_cg_want<<<gc, 128, 0, st>>>(s, rrnew, R);
      AGP_CUDA(cudaMemcpyAsync(want.data(), s.want, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
      AGP_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int v : want) any = any || v == 1;
      if (any) {   // r = b - K x for every column that asked (or would soon)
        for (int part = 0; part < (sizeof(T) == 4 ? 2 : 1); ++part) {
          k_cg_xsplit<T><<<gb, 256, 0, st>>>(ws.x, ws.pt, part, n * R);
          AGP_TRY(agp_matvec(pl, ws.pt, R, ws.q, R, R, 1, st));
          k_cg_replace<T><<<gb, 256, 0, st>>>(ws.r, B, ldb, ws.q, s.want, part, n, R);
          pl->launches[3] += 2;
        }
        AGP_TRY(col_dot(ws.r, R, ws.r, R, n, R, ws.partial, rrnew, st, pl));
        k_cg_replaced<<<gc, 128, 0, st>>>(s, rrnew, R);
        pl->launches[3] += 1;
      } else {
        AGP_CUDA(cudaMemsetAsync(s.want, 0, sizeof(int) * R, st));
      }
    }
    if (pcon) {
      AGP_TRY(apply_pc());
      AGP_TRY(col_dot(ws.r, R, ws.z, R, n, R, ws.partial, s.rznew, st, pl));
    }
    k_cg_beta<<<gc, 128, 0, st>>>(s, rrnew, it, R);
    k_cg_p<T><<<gb, 256, 0, st>>>(ws.p, ws.pt, pcon ? ws.z : ws.r, s.beta, s.active, n, R);
    pl->launches[3] += 2;
    AGP_CUDA(cudaGetLastError());
    if (check_every > 0 && ((it + 1) % check_every == 0) && it + 1 < maxall) {
      AGP_CUDA(cudaMemcpyAsync(act.data(), s.active, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
      AGP_CUDA(cudaStreamSynchronize(st));
      bool any = false;
      for (int v : act) any = any || v;
      if (!any) break;
    }
  }
  k_copy_block<double, T><<<gb, 256, 0, st>>>(ws.x, R, X, ldx, n, R);
  pl->launches[3] += 1;
  return cuda_status(cudaGetLastError(), "cg_run");
}

template <typename T>
agp_status pcg_t(agp_plan_s* pl, const T* B, int64_t ldb, T* X, int64_t ldx, int R, double rtol,
                 int maxit, int n_landmarks, int* iters, double* relres, cudaStream_t st,
                 const Afn* afn = nullptr) {
  Precond pc;
  struct Release {
    Precond* p;
    ~Release() { precond_free(p); }
  } release{&pc};
  if (n_landmarks > 0) AGP_TRY(precond_build<T>(pl, n_landmarks, R, &pc, st));
  Workspace<T> ws;
  std::vector<int> mi(R, maxit);
  std::vector<double> tl(R, rtol);
  AGP_TRY(cg_run<T>(pl, B, ldb, X, ldx, R, mi, tl, 5, ws, st, n_landmarks > 0 ? &pc : nullptr,
                    afn, true));
  std::vector<int> it(R);
  std::vector<double> rel(R);
  AGP_CUDA(cudaMemcpyAsync(it.data(), ws.iscal + R, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaMemcpyAsync(rel.data(), ws.scal + 5 * R, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  bool ok = true;
  for (int c = 0; c < R; ++c) {
    if (iters) iters[c] = it[c];
    if (relres) relres[c] = rel[c];
    ok = ok && rel[c] <= rtol;
  }
  if (!ok) return set_error(AGP_NOT_CONVERGED, "CG stopped at maxit above the tolerance");
  return AGP_OK;
}

// Rademacher probes (Hutchinson's estimator, Sec. 1) from the counter-based
// SplitMix64 generator (Steele, Lea and Flood, OOPSLA 2014): entry (i, c) of
// an n x R block is +1 when the top bit of output i R + c is 0, else -1;
// output j mixes the state seed + (j + 1) g, g = 0x9E3779B97F4A7C15.
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t j) {
  uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_rademacher(T* __restrict__ Z, int64_t ldz, int64_t n, int R, uint64_t seed) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t i = e / R;
  const int c = (int)(e - i * R);
  Z[i * ldz + c] = (splitmix64_out(seed, (uint64_t)e) >> 63) ? T(-1) : T(1);
}

// Lanczos breakdown floor of the NLML estimators (Sec. 1, SLQ by CG-Lanczos):
// a column whose relative residual has fallen to this level has reached an
// invariant Krylov subspace to working precision; its Lanczos matrix ends
// there (the Gauss quadrature is then exact to that precision), since the
// coefficients of further steps would be ratios of rounding-level residual
// norms and change from run to run with the order of the atomic additions.
template <typename T>
constexpr double lanczos_floor() {
  return sizeof(T) == 4 ? 1e-6 : 1e-12;
}

template <typename T>
agp_status nlml_t(agp_plan_s* pl, const T* Y, const T* Z, int64_t ldz, int nz, int steps,
                  double rtol, int maxit, double* nlml, double* grad, cudaStream_t st) {
  const int64_t n = pl->n;
  const int R = 1 + nz;
  T *B = nullptr, *Xs = nullptr, *D = nullptr;
  double* dots = nullptr;
  AGP_CUDA(cudaMallocAsync(&B, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Xs, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&D, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&dots, sizeof(double) * 4 * R, st));
  struct Free {
    void* a[4];
    cudaStream_t st;
    ~Free() {
      for (void* p : a) cudaFreeAsync(p, st);
    }
  } fr{{B, Xs, D, dots}, st};
  k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Y, 1, B, R, n, 1);
  k_copy_block<T, T><<<nblk(n * nz, 256), 256, 0, st>>>(Z, ldz, B + 1, R, n, nz);
  pl->launches[3] += 2;
  AGP_CUDA(cudaGetLastError());
  std::vector<int> mi(R, steps);
  std::vector<double> tl(R, lanczos_floor<T>());
  if (rtol > 0) {
    mi[0] = maxit;
    tl[0] = rtol;
  }
  {
    Workspace<T> ws;
    AGP_TRY(cg_run<T>(pl, B, R, Xs, R, R, mi, tl, rtol > 0 ? 5 : 0, ws, st));
    // y^T alpha and the SLQ quadratures of the probes
    AGP_TRY(col_dot(B, R, Xs, R, n, 1, ws.partial, dots, st, pl));
    k_slq_logdet<<<nblk(nz, kSlqThreads), kSlqThreads, 0, st>>>(ws.ahist, ws.bhist, ws.iscal + R, ws.scal + R, R, 1,
                                              dots + R);
    pl->launches[3] += 1;
    AGP_CUDA(cudaGetLastError());
  }
  std::vector<double> h(R + 1);
  AGP_CUDA(cudaMemcpyAsync(h.data(), dots, sizeof(double) * (R), cudaMemcpyDeviceToHost, st));
  // dots[R + c] holds the quadrature of column c (c >= 1)
  std::vector<double> quad(R);
  AGP_CUDA(cudaMemcpyAsync(quad.data(), dots + R, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  double logdet = 0.0;
  for (int c = 1; c < R; ++c) logdet += quad[c];
  logdet /= nz;
  *nlml = 0.5 * (h[0] + logdet + (double)n * std::log(2.0 * M_PI));

  // gradient: 1/2 (-alpha^T dK alpha + (1/nz) sum_i u_i^T dK z_i), Xs = [alpha, u_1..u_nz]
  const agp_param ths[3] = {AGP_D_ELL, AGP_D_SIGMA_F, AGP_D_SIGMA_EPS};
  for (int k = 0; k < 3; ++k) {
    // dK applied to [alpha, z_1..z_nz]: build that block in D's scratch (reuse B)
    k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Xs, R, B, R, n, 1);
    pl->launches[3] += 1;
    AGP_TRY(agp_deriv_matvec(pl, ths[k], B, R, D, R, R, st));
    double* part = nullptr;
    AGP_CUDA(cudaMallocAsync(&part, sizeof(double) * kMaxDotBlocks * R, st));
    agp_status s = col_dot(Xs, R, D, R, n, R, part, dots + 2 * R, st, pl);
    cudaFreeAsync(part, st);
    if (s != AGP_OK) return s;
    std::vector<double> g(R);
    AGP_CUDA(cudaMemcpyAsync(g.data(), dots + 2 * R, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    double tr = 0.0;
    for (int c = 1; c < R; ++c) tr += g[c];
    grad[k] = 0.5 * (-g[0] + tr / nz);
  }
  // A non-positive Ritz value makes log theta undefined: the truncated
  // operator (no boundary smoothing, Sec. 3.1) is indefinite at these
  // hyperparameters. The gradient estimate above does not use logarithms.
  if (!std::isfinite(*nlml))
    return set_error(AGP_ENAN, "SLQ met a non-positive Ritz value: K_hat is indefinite here");
  return AGP_OK;
}

// Preconditioned NLML estimate and gradient, Sec. 1 eqs. (1.3)-(1.5), with the
// landmark preconditioner M = B K_LL^{-1} B^T + sigma_eps^2 I of Sec. 2.3:
//   nlml = 1/2 (y^T alpha + log det M + (1/nz) sum_i q_i + n log 2 pi),
//   q_i  = (z_i^T M^{-1} z_i) e_1^T log(T_i) e_1  (SLQ of M^{-1/2} K_hat M^{-1/2}),
//   grad = 1/2 (-alpha^T dK alpha + tr(M^{-1} dM) + (1/nz) sum_i (u_i^T dK p_i - p_i^T dM p_i)),
// z_i = sigma_eps wn_i + B C^{-T} wk_i (covariance M, C C^T = K_LL), T_i from
// `steps` PCG steps on K_hat x = z_i, u_i the PCG iterate, p_i = M^{-1} z_i.
// The k x k algebra runs on the host in FP64: with G = sigma^2 K_LL + B^T B,
//   log det M = (n - k) log sigma^2 + log det G - log det K_LL,
//   tr(M^{-1}) = (n - k + sigma^2 tr(G^{-1} K_LL)) / sigma^2,
//   tr(M^{-1} dM/dell) = 2 tr(G^{-1} B^T B') - tr(K'_LL K_LL^{-1}) + sigma^2 tr(K'_LL G^{-1}),
// (B' = dB/dell; for sigma_f, B' = (2/sigma_f) B and K'_LL = (2/sigma_f)(K_LL - delta I)
// with the jitter delta held fixed), dM/dsigma_eps = 2 sigma_eps I.
template <typename T>
agp_status nlml_pc_t(agp_plan_s* pl, const T* Y, const T* Wn, int64_t ldwn, const double* Wk_h,
                     int nz, int n_landmarks, int steps, double rtol, int maxit, double* nlml,
                     double* grad, cudaStream_t st) {
  const int64_t n = pl->n;
  const int R = 1 + nz;
  const double sig = pl->sigma_eps, s2 = sig * sig, sf = pl->sigma_f;
  Precond pc;
  struct Release {
    Precond* p;
    ~Release() { precond_free(p); }
  } release{&pc};
  PrecondNlml ex;
  AGP_TRY(precond_build<T>(pl, n_landmarks, R, &pc, st, &ex));
  const int k = pc.k;
  auto tr_prod = [&](const std::vector<double>& A, const std::vector<double>& Bm) {
    double t = 0.0;   // tr(A Bm) = sum_ij A_ij Bm_ji
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) t += A[(size_t)i * k + j] * Bm[(size_t)j * k + i];
    return t;
  };
  // probes: Tk = C^{-T} Wk (back substitution with the lower factor C)
  std::vector<double> Tk((size_t)k * nz);
  for (int r = 0; r < nz; ++r)
    for (int j = k - 1; j >= 0; --j) {
      double v = Wk_h[(size_t)j * nz + r];
      for (int i = j + 1; i < k; ++i) v -= ex.Kchol[(size_t)i * k + j] * Tk[(size_t)i * nz + r];
      Tk[(size_t)j * nz + r] = v / ex.Kchol[(size_t)j * k + j];
    }
  T *Bblk = nullptr, *Xs = nullptr, *Din = nullptr, *Dout = nullptr;
  double *Tk_d = nullptr, *Zd = nullptr, *Pd = nullptr, *dots = nullptr, *part = nullptr;
  AGP_CUDA(cudaMallocAsync(&Bblk, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Xs, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Din, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Dout, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Tk_d, sizeof(double) * k * nz, st));
  AGP_CUDA(cudaMallocAsync(&Zd, sizeof(double) * n * nz, st));
  AGP_CUDA(cudaMallocAsync(&Pd, sizeof(double) * n * nz, st));
  AGP_CUDA(cudaMallocAsync(&dots, sizeof(double) * 4 * R, st));
  AGP_CUDA(cudaMallocAsync(&part, sizeof(double) * kMaxDotBlocks * R, st));
  struct Free {
    void* a[9];
    cudaStream_t st;
    ~Free() {
      for (void* p : a) cudaFreeAsync(p, st);
    }
  } fr{{Bblk, Xs, Din, Dout, Tk_d, Zd, Pd, dots, part}, st};
  AGP_CUDA(cudaMemcpyAsync(Tk_d, Tk.data(), sizeof(double) * k * nz, cudaMemcpyHostToDevice, st));
  k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Y, 1, Bblk, R, n, 1);
  pl->launches[3] += 1;
  AGP_TRY(precond_affine<T>(pc, sig, Wn, ldwn, Tk_d, nz, Bblk + 1, R, st));
  // PCG on [y, z_1..z_nz]: probes run exactly `steps` steps (their coefficients
  // give the Lanczos matrices), y to rtol when rtol > 0
  std::vector<int> mi(R, steps);
  std::vector<double> tl(R, lanczos_floor<T>());
  if (rtol > 0) {
    mi[0] = maxit;
    tl[0] = rtol;
  }
  std::vector<double> h(2 * R);
  {
    Workspace<T> ws;
    AGP_TRY(cg_run<T>(pl, Bblk, R, Xs, R, R, mi, tl, rtol > 0 ? 5 : 0, ws, st, &pc));
    AGP_TRY(col_dot(Bblk, R, Xs, R, n, 1, ws.partial, dots, st, pl));
    k_slq_logdet<<<nblk(nz, kSlqThreads), kSlqThreads, 0, st>>>(ws.ahist, ws.bhist, ws.iscal + R,
                                                                 ws.rz0, R, 1, dots + R);
    pl->launches[3] += 1;
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(h.data(), dots, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
  }
  double quad = 0.0;
  for (int c = 1; c < R; ++c) quad += h[R + c];
  const double logdet_M = (double)(n - k) * std::log(s2) + ex.logdet_G - ex.logdet_K;
  *nlml = 0.5 * (h[0] + logdet_M + quad / nz + (double)n * std::log(2.0 * M_PI));

  // p_i = M^{-1} z_i and the small-dimensional terms
  k_copy_block<T, double><<<nblk(n * nz, 256), 256, 0, st>>>(Bblk + 1, R, Zd, nz, n, nz);
  pl->launches[3] += 1;
  AGP_TRY(precond_apply<T>(pc, Zd, Pd, nz, st));
  std::vector<double> A((size_t)k * nz), E((size_t)k * nz), pp(nz);
  AGP_TRY(precond_bt<T>(pc, 0, Pd, nz, A.data(), st));
  AGP_TRY(precond_bt<T>(pc, 1, Pd, nz, E.data(), st));
  AGP_TRY(col_dot(Pd, nz, Pd, nz, n, nz, part, dots, st, pl));
  AGP_CUDA(cudaMemcpyAsync(pp.data(), dots, sizeof(double) * nz, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  const double tr_gk = tr_prod(ex.Ginv, ex.K);
  const double tr_minv = ((double)(n - k) + s2 * tr_gk) / s2;
  double tr_kinv = 0.0, tr_ginv = 0.0;
  for (int i = 0; i < k; ++i) {
    tr_kinv += ex.Kinv[(size_t)i * k + i];
    tr_ginv += ex.Ginv[(size_t)i * k + i];
  }
  // sigma_f: dB = (2/sigma_f) B and dK_LL = (2/sigma_f)(K - delta I) with the
  // jitter delta held fixed
  const double tr_dm[3] = {
      2.0 * tr_prod(ex.Ginv, ex.BtBder) - tr_prod(ex.Kder, ex.Kinv) + s2 * tr_prod(ex.Kder, ex.Ginv),
      (2.0 / sf) * ((double)k - s2 * tr_gk + ex.delta * tr_kinv - s2 * ex.delta * tr_ginv),
      2.0 * sig * tr_minv};
  // p_i^T dM p_i with a = B^T p_i, e = B'^T p_i, v = K_LL^{-1} a
  std::vector<double> pdp[3] = {std::vector<double>(nz), std::vector<double>(nz),
                                std::vector<double>(nz)};
  std::vector<double> v(k);
  for (int r = 0; r < nz; ++r) {
    for (int i = 0; i < k; ++i) {
      double t = 0.0;
      for (int j = 0; j < k; ++j) t += ex.Kinv[(size_t)i * k + j] * A[(size_t)j * nz + r];
      v[i] = t;
    }
    double va = 0.0, ve = 0.0, vkv = 0.0, vv = 0.0;
    for (int i = 0; i < k; ++i) {
      va += v[i] * A[(size_t)i * nz + r];
      vv += v[i] * v[i];
      ve += v[i] * E[(size_t)i * nz + r];
      double t = 0.0;
      for (int j = 0; j < k; ++j) t += ex.Kder[(size_t)i * k + j] * v[j];
      vkv += v[i] * t;
    }
    pdp[0][r] = 2.0 * ve - vkv;
    pdp[1][r] = (2.0 / sf) * (va + ex.delta * vv);
    pdp[2][r] = 2.0 * sig * pp[r];
  }
  // dK applied to [alpha, p_1..p_nz], dotted with [alpha, u_1..u_nz]
  k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Xs, R, Din, R, n, 1);
  k_copy_block<double, T><<<nblk(n * nz, 256), 256, 0, st>>>(Pd, nz, Din + 1, R, n, nz);
  pl->launches[3] += 2;
  const agp_param ths[3] = {AGP_D_ELL, AGP_D_SIGMA_F, AGP_D_SIGMA_EPS};
  for (int t = 0; t < 3; ++t) {
    AGP_TRY(agp_deriv_matvec(pl, ths[t], Din, R, Dout, R, R, st));
    AGP_TRY(col_dot(Xs, R, Dout, R, n, R, part, dots, st, pl));
    std::vector<double> g(R);
    AGP_CUDA(cudaMemcpyAsync(g.data(), dots, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    double smean = 0.0;
    for (int r = 0; r < nz; ++r) smean += g[1 + r] - pdp[t][r];
    grad[t] = 0.5 * (-g[0] + tr_dm[t] + smean / nz);
  }
  if (!std::isfinite(*nlml))
    return set_error(AGP_ENAN, "SLQ met a non-positive Ritz value: K_hat is indefinite here");
  return AGP_OK;
}

// out[j][r] = X[rows_j][r] (FP64 [cnt][R] from the plan precision [n][ldx])
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ X, int64_t ldx, const int32_t* __restrict__ rows,
                              int64_t cnt, int R, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cnt * R) return;
  const int64_t j = e / R;
  out[e] = (double)X[(int64_t)rows[j] * ldx + (e - j * R)];
}

// AFN probes: Z[F_a][r] = sum_j W[a][j] wL[j][r] + y[a][r] (a warp per row,
// wL staged in shared memory), Z[L_j][r] = zL[j][r]; Z in the plan precision
template <typename T>
__global__ void __launch_bounds__(256)
k_afn_probe_f(const double* __restrict__ W, const int32_t* __restrict__ F, int64_t m, int k, int nz,
              const double* __restrict__ wL, const double* __restrict__ y, T* __restrict__ Z,
              int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sw = reinterpret_cast<double*>(smem_raw);
  for (int e = threadIdx.x; e < k * nz; e += blockDim.x) sw[e] = wL[e];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  if (lane >= nz) return;
  for (int64_t a = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; a < m; a += (int64_t)gridDim.x * 8) {
    const double* wr = W + a * k;
    double s = y[a * nz + lane];
    for (int j = 0; j < k; ++j) s = fma(wr[j], sw[j * nz + lane], s);
    Z[(int64_t)F[a] * ldz + lane] = (T)s;
  }
}

template <typename T>
__global__ void k_scatter_rows(const double* __restrict__ src, const int32_t* __restrict__ rows,
                               int cnt, int R, T* __restrict__ Z, int64_t ldz) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cnt * R) return;
  const int j = e / R;
  Z[(int64_t)rows[j] * ldz + (e - j * R)] = (T)src[e];
}

// x = K_LL^{-1} b for the columns of b (host [k][R]) with the lower factor C
void chol_solve_host(const std::vector<double>& C, int k, int R, std::vector<double>& b) {
  for (int r = 0; r < R; ++r) {
    for (int i = 0; i < k; ++i) {
      double v = b[(size_t)i * R + r];
      for (int j = 0; j < i; ++j) v -= C[(size_t)i * k + j] * b[(size_t)j * R + r];
      b[(size_t)i * R + r] = v / C[(size_t)i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double v = b[(size_t)i * R + r];
      for (int j = i + 1; j < k; ++j) v -= C[(size_t)j * k + i] * b[(size_t)j * R + r];
      b[(size_t)i * R + r] = v / C[(size_t)i * k + i];
    }
  }
}

// NLML estimate and gradient with the additive AFN preconditioner (Sec. 1
// eqs. (1.3)-(1.5), M of Sec. 2.3 as built by afn_build): the estimator of
// nlml_pc_t with
//   probes     z_L = C w_L, z_F = W w_L + G^{-1} w_F  (covariance M),
//   log det M  from the factors, tr(M^{-1} dM) = d log det M / dtheta =
//              tr(K_LL^{-1} dK_LL) + sum_t G_t^T dS G_t,
//   p^T dM p = 2 (dX^T w).z_L + q_L^T dK_LL q_L - 2 u^T (dG t)
// for p = M^{-1} z, where X = K_FL K_LL^{-1}, q_L = K_LL^{-1} z_L, and t =
// z_F - X z_L, u = G t, w = G^T u = p_F are the apply's intermediates;
// dX^T w = K_LL^{-1} (dK_LF w - dK_LL X^T w) with X^T w = C^{-T} W^T w.
template <typename T>
agp_status nlml_afn_t(agp_plan_s* pl, Afn* af, const T* Y, const T* Wn, int64_t ldwn, int nz,
                      int steps, double rtol, int maxit, double* nlml, double* grad,
                      cudaStream_t st) {
  const int64_t n = pl->n, m = af->m;
  const int R = 1 + nz, k = af->k;
  const double sig = pl->sigma_eps, s2 = sig * sig, sf = pl->sigma_f;
  AGP_TRY(afn_build_derivs<T>(pl, af, st));
  const std::vector<double>& C = af->C_h;
  T *Bblk = nullptr, *Xs = nullptr, *Din = nullptr, *Dout = nullptr;
  double *wF = nullptr, *yF = nullptr, *wL = nullptr, *Zd = nullptr, *Pd = nullptr, *dots = nullptr,
         *part = nullptr, *tmp = nullptr;
  AGP_CUDA(cudaMallocAsync(&Bblk, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Xs, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Din, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&Dout, sizeof(T) * n * R, st));
  AGP_CUDA(cudaMallocAsync(&wF, sizeof(double) * std::max<int64_t>(1, m) * nz, st));
  AGP_CUDA(cudaMallocAsync(&yF, sizeof(double) * std::max<int64_t>(1, m) * nz, st));
  AGP_CUDA(cudaMallocAsync(&tmp, sizeof(double) * std::max<int64_t>(1, m) * nz, st));
  AGP_CUDA(cudaMallocAsync(&wL, sizeof(double) * k * nz, st));
  AGP_CUDA(cudaMallocAsync(&Zd, sizeof(double) * n * nz, st));
  AGP_CUDA(cudaMallocAsync(&Pd, sizeof(double) * n * nz, st));
  AGP_CUDA(cudaMallocAsync(&dots, sizeof(double) * 4 * R, st));
  AGP_CUDA(cudaMallocAsync(&part, sizeof(double) * kMaxDotBlocks * R, st));
  struct Free {
    void* a[12];
    cudaStream_t st;
    ~Free() {
      for (void* p : a) cudaFreeAsync(p, st);
    }
  } fr{{Bblk, Xs, Din, Dout, wF, yF, tmp, wL, Zd, Pd, dots, part}, st};
  // probes
  std::vector<double> wLh((size_t)k * nz);
  k_gather_rows<T><<<nblk((int64_t)k * nz, 256), 256, 0, st>>>(Wn, ldwn, af->L, k, nz, wL);
  AGP_CUDA(cudaMemcpyAsync(wLh.data(), wL, sizeof(double) * k * nz, cudaMemcpyDeviceToHost, st));
  k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Y, 1, Bblk, R, n, 1);
  pl->launches[3] += 2;
  if (m > 0) {
    k_gather_rows<T><<<nblk(m * nz, 256), 256, 0, st>>>(Wn, ldwn, af->F, m, nz, wF);
    AGP_TRY(afn_trsv(*af, wF, yF, nz, st));
    const size_t smem = sizeof(double) * (size_t)k * nz;
    AGP_CUDA(cudaFuncSetAttribute(k_afn_probe_f<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * kMaxLandmarkSet * 32)));
    const unsigned blocks = (unsigned)std::min<int64_t>(nblk(m, 8), 152 * 16);
    k_afn_probe_f<T><<<blocks, 256, smem, st>>>(af->W, af->F, m, k, nz, wL, yF, Bblk + 1, R);
    pl->launches[3] += (int64_t)af->lvl_off.size() + 1;
  }
  AGP_CUDA(cudaStreamSynchronize(st));
  std::vector<double> zLh((size_t)k * nz, 0.0);
  for (int i = 0; i < k; ++i)
    for (int r = 0; r < nz; ++r) {
      double v = 0.0;
      for (int j = 0; j <= i; ++j) v += C[(size_t)i * k + j] * wLh[(size_t)j * nz + r];
      zLh[(size_t)i * nz + r] = v;
    }
  AGP_CUDA(cudaMemcpyAsync(wL, zLh.data(), sizeof(double) * k * nz, cudaMemcpyHostToDevice, st));
  k_scatter_rows<T><<<nblk((int64_t)k * nz, 128), 128, 0, st>>>(wL, af->L, k, nz, Bblk + 1, R);
  pl->launches[3] += 1;
  AGP_CUDA(cudaGetLastError());
  // PCG-Lanczos on [y, z_1..z_nz]
  std::vector<int> mi(R, steps);
  std::vector<double> tl(R, lanczos_floor<T>());
  if (rtol > 0) {
    mi[0] = maxit;
    tl[0] = rtol;
  }
  std::vector<double> h(2 * R);
  {
    Workspace<T> ws;
    AGP_TRY(cg_run<T>(pl, Bblk, R, Xs, R, R, mi, tl, rtol > 0 ? 5 : 0, ws, st, nullptr, af));
    AGP_TRY(col_dot(Bblk, R, Xs, R, n, 1, ws.partial, dots, st, pl));
    k_slq_logdet<<<nblk(nz, kSlqThreads), kSlqThreads, 0, st>>>(ws.ahist, ws.bhist, ws.iscal + R,
                                                                 ws.rz0, R, 1, dots + R);
    pl->launches[3] += 1;
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(h.data(), dots, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
  }
  double quad = 0.0;
  for (int c = 1; c < R; ++c) quad += h[R + c];
  *nlml = 0.5 * (h[0] + af->logdet + quad / nz + (double)n * std::log(2.0 * M_PI));

  // p = M^{-1} z (z as rounded to the plan precision); the apply leaves t, u
  // and w = p_F in af->t, af->u, af->w
  k_copy_block<T, double><<<nblk(n * nz, 256), 256, 0, st>>>(Bblk + 1, R, Zd, nz, n, nz);
  pl->launches[3] += 1;
  AGP_TRY(afn_apply(*af, Zd, nz, Pd, nz, nz, st));
  std::vector<double> zL((size_t)k * nz), WTw((size_t)k * nz), DTw((size_t)k * nz);
  k_gather_rows<double><<<nblk((int64_t)k * nz, 256), 256, 0, st>>>(Zd, nz, af->L, k, nz, wL);
  AGP_CUDA(cudaMemcpyAsync(zL.data(), wL, sizeof(double) * k * nz, cudaMemcpyDeviceToHost, st));
  AGP_TRY(afn_wt(*af, af->W, af->w, nz, WTw.data(), st));
  AGP_TRY(afn_wt(*af, af->Dl, af->w, nz, DTw.data(), st));
  // -2 u^T (dG_theta t), per column
  std::vector<double> udgt[3];
  for (int th = 0; th < 3; ++th) {
    udgt[th].assign(nz, 0.0);
    if (m == 0) continue;
    AGP_TRY(afn_dg_apply(*af, th, af->t, tmp, nz, st));
    AGP_TRY(col_dot(af->u, nz, tmp, nz, m, nz, part, dots, st, pl));
    AGP_CUDA(cudaMemcpyAsync(udgt[th].data(), dots, sizeof(double) * nz, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
  }
  // host k x k algebra
  std::vector<double> qL = zL;
  chol_solve_host(C, k, nz, qL);                       // K_LL^{-1} z_L
  std::vector<double> XTw((size_t)k * nz);             // C^{-T} W^T w
  for (int r = 0; r < nz; ++r)
    for (int i = k - 1; i >= 0; --i) {
      double v = WTw[(size_t)i * nz + r];
      for (int j = i + 1; j < k; ++j) v -= C[(size_t)j * k + i] * XTw[(size_t)j * nz + r];
      XTw[(size_t)i * nz + r] = v / C[(size_t)i * k + i];
    }
  std::vector<double> KinvXTw = XTw;
  chol_solve_host(C, k, nz, KinvXTw);
  // dX^T w for ell: K_LL^{-1} (C (Dl^T w) - dK_LL X^T w)
  std::vector<double> dxw((size_t)k * nz);
  for (int i = 0; i < k; ++i)
    for (int r = 0; r < nz; ++r) {
      double v = 0.0;
      for (int j = 0; j <= i; ++j) v += C[(size_t)i * k + j] * DTw[(size_t)j * nz + r];
      for (int j = 0; j < k; ++j) v -= af->dKLL_h[(size_t)i * k + j] * XTw[(size_t)j * nz + r];
      dxw[(size_t)i * nz + r] = v;
    }
  chol_solve_host(C, k, nz, dxw);
  // K_LL^{-1} (host, from C^{-1}) for the traces
  const std::vector<double>& Ci = af->Ci_h;
  double tr_kinv = 0.0, tr_kinv_dk = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double v = 0.0;   // (C^{-T} C^{-1})_ij
      for (int q = std::max(i, j); q < k; ++q) v += Ci[(size_t)q * k + i] * Ci[(size_t)q * k + j];
      if (i == j) tr_kinv += v;
      tr_kinv_dk += v * af->dKLL_h[(size_t)j * k + i];
    }
  const double tr_dm[3] = {tr_kinv_dk + af->quad_sum[0],
                           (2.0 / sf) * ((double)k - s2 * tr_kinv) + af->quad_sum[1],
                           2.0 * sig * tr_kinv + af->quad_sum[2]};
  std::vector<double> pdp[3] = {std::vector<double>(nz), std::vector<double>(nz),
                                std::vector<double>(nz)};
  for (int r = 0; r < nz; ++r) {
    double t1[3] = {0, 0, 0}, qkq = 0.0, qdq = 0.0, qq = 0.0;
    for (int i = 0; i < k; ++i) {
      const double zl = zL[(size_t)i * nz + r], ql = qL[(size_t)i * nz + r];
      t1[0] += dxw[(size_t)i * nz + r] * zl;
      t1[1] += (2.0 / sf) * s2 * KinvXTw[(size_t)i * nz + r] * zl;
      t1[2] += -2.0 * sig * KinvXTw[(size_t)i * nz + r] * zl;
      qq += ql * ql;
      double a = 0.0, b = 0.0;
      for (int j = 0; j < k; ++j) {
        a += af->KLL_h[(size_t)i * k + j] * qL[(size_t)j * nz + r];
        b += af->dKLL_h[(size_t)i * k + j] * qL[(size_t)j * nz + r];
      }
      qkq += ql * a;
      qdq += ql * b;
    }
    pdp[0][r] = 2.0 * t1[0] + qdq - 2.0 * udgt[0][r];
    pdp[1][r] = 2.0 * t1[1] + (2.0 / sf) * (qkq - s2 * qq) - 2.0 * udgt[1][r];
    pdp[2][r] = 2.0 * t1[2] + 2.0 * sig * qq - 2.0 * udgt[2][r];
  }
  // dK applied to [alpha, p_1..p_nz], dotted with [alpha, u_1..u_nz]
  k_copy_block<T, T><<<nblk(n, 256), 256, 0, st>>>(Xs, R, Din, R, n, 1);
  k_copy_block<double, T><<<nblk(n * nz, 256), 256, 0, st>>>(Pd, nz, Din + 1, R, n, nz);
  pl->launches[3] += 2;
  const agp_param ths[3] = {AGP_D_ELL, AGP_D_SIGMA_F, AGP_D_SIGMA_EPS};
  for (int t = 0; t < 3; ++t) {
    AGP_TRY(agp_deriv_matvec(pl, ths[t], Din, R, Dout, R, R, st));
    AGP_TRY(col_dot(Xs, R, Dout, R, n, R, part, dots, st, pl));
    std::vector<double> g(R);
    AGP_CUDA(cudaMemcpyAsync(g.data(), dots, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    double smean = 0.0;
    for (int r = 0; r < nz; ++r) smean += g[1 + r] - pdp[t][r];
    grad[t] = 0.5 * (-g[0] + tr_dm[t] + smean / nz);
  }
  if (!std::isfinite(*nlml))
    return set_error(AGP_ENAN, "SLQ met a non-positive Ritz value: K_hat is indefinite here");
  return AGP_OK;
}

}  // namespace
}  // namespace agp

using namespace agp;

extern "C" {

agp_status agp_pcg_solve(agp_plan pl, const void* B, int64_t ldb, void* Xsol, int64_t ldx, int R,
                         double rtol, int maxit, int n_landmarks, int* iters, double* relres,
                         void* stream) {
  if (!pl || !B || !Xsol || R < 1 || ldb < R || ldx < R || maxit < 0 || !(rtol >= 0))
    return set_error(AGP_EINVAL, "bad arguments");
  if (n_landmarks < 0 || n_landmarks > kMaxLandmarks || (n_landmarks > 0 && R > 32))
    return set_error(AGP_EINVAL, "n_landmarks must be in [0, 480] (and R <= 32 when > 0)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const agp_status s =
      pl->prec == AGP_F32
          ? pcg_t<float>(pl, (const float*)B, ldb, (float*)Xsol, ldx, R, rtol, maxit, n_landmarks,
                         iters, relres, st)
          : pcg_t<double>(pl, (const double*)B, ldb, (double*)Xsol, ldx, R, rtol, maxit,
                          n_landmarks, iters, relres, st);
  return with_timeout_check(pl, s, st);
}

agp_status agp_afn_create(agp_afn* out, agp_plan pl, int n_landmarks, int fill, void* stream) {
  if (!out) return set_error(AGP_EINVAL, "bad arguments");
  *out = nullptr;
  if (!pl || n_landmarks < 1 || n_landmarks > kMaxLandmarks || fill < 1 || fill > kAfnMaxFill)
    return set_error(AGP_EINVAL, "n_landmarks must be in [1, 480] and fill in [1, 128]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Afn* af = new Afn();
  const agp_status s = pl->prec == AGP_F32 ? afn_build<float>(pl, n_landmarks, fill, 32, af, st)
                                           : afn_build<double>(pl, n_landmarks, fill, 32, af, st);
  if (s != AGP_OK) {
    cudaStreamSynchronize(st);
    afn_free(af);
    delete af;
    return s;
  }
  *out = reinterpret_cast<agp_afn>(af);
  return AGP_OK;
}

agp_status agp_afn_destroy(agp_afn afn) {
  if (!afn) return AGP_OK;
  Afn* af = reinterpret_cast<Afn*>(afn);
  afn_free(af);   // cudaFree waits for the device
  delete af;
  return AGP_OK;
}

agp_status agp_afn_apply(agp_afn afn, const double* V, int64_t ldv, double* Y, int64_t ldy, int R,
                         void* stream) {
  if (!afn || !V || !Y || R < 1 || R > 32 || ldv < R || ldy < R)
    return set_error(AGP_EINVAL, "bad arguments");
  return afn_apply(*reinterpret_cast<const Afn*>(afn), V, ldv, Y, ldy, R,
                   static_cast<cudaStream_t>(stream));
}

agp_status agp_afn_info(agp_afn afn, int* n_landmarks, int64_t* nnz, double* logdet) {
  if (!afn) return set_error(AGP_EINVAL, "bad arguments");
  const Afn* af = reinterpret_cast<const Afn*>(afn);
  if (n_landmarks) *n_landmarks = af->k;
  if (nnz) *nnz = af->nnz;
  if (logdet) *logdet = af->logdet;
  return AGP_OK;
}

agp_status agp_afn_pattern(agp_afn afn, int32_t* landmarks, int32_t* J, void* stream) {
  if (!afn) return set_error(AGP_EINVAL, "bad arguments");
  return afn_pattern(*reinterpret_cast<const Afn*>(afn), landmarks, J,
                     static_cast<cudaStream_t>(stream));
}

agp_status agp_pcg_solve_afn(agp_plan pl, agp_afn afn, const void* B, int64_t ldb, void* Xsol,
                             int64_t ldx, int R, double rtol, int maxit, int* iters,
                             double* relres, void* stream) {
  if (!pl || !afn || !B || !Xsol || R < 1 || R > 32 || ldb < R || ldx < R || maxit < 0 ||
      !(rtol >= 0))
    return set_error(AGP_EINVAL, "bad arguments");
  const Afn* af = reinterpret_cast<const Afn*>(afn);
  if (af->n != pl->n || af->ell != pl->ell || af->sigma_f != pl->sigma_f ||
      af->sigma_eps != pl->sigma_eps || af->kernel != (int)pl->kernel)
    return set_error(AGP_EINVAL, "the AFN preconditioner was built for other hyperparameters");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const agp_status s =
      pl->prec == AGP_F32
          ? pcg_t<float>(pl, (const float*)B, ldb, (float*)Xsol, ldx, R, rtol, maxit, 0, iters,
                         relres, st, af)
          : pcg_t<double>(pl, (const double*)B, ldb, (double*)Xsol, ldx, R, rtol, maxit, 0, iters,
                          relres, st, af);
  return with_timeout_check(pl, s, st);
}

agp_status agp_nlml_grad_afn(agp_plan pl, agp_afn afn, const void* Y, const void* Wn,
                             int64_t ldwn, int nz, int lanczos_steps, double rtol, int maxit,
                             double* nlml, double* grad, void* stream) {
  if (!pl || !afn || !Y || !Wn || !nlml || !grad || nz < 1 || nz > 31 || ldwn < nz ||
      lanczos_steps < 1 || lanczos_steps > kMaxLanczos || !(rtol >= 0) || (rtol > 0 && maxit < 1))
    return set_error(AGP_EINVAL, "bad arguments");
  Afn* af = reinterpret_cast<Afn*>(afn);
  if (af->n != pl->n || af->ell != pl->ell || af->sigma_f != pl->sigma_f ||
      af->sigma_eps != pl->sigma_eps || af->kernel != (int)pl->kernel)
    return set_error(AGP_EINVAL, "the AFN preconditioner was built for other hyperparameters");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const agp_status s =
      pl->prec == AGP_F32
          ? nlml_afn_t<float>(pl, af, (const float*)Y, (const float*)Wn, ldwn, nz, lanczos_steps,
                              rtol, maxit, nlml, grad, st)
          : nlml_afn_t<double>(pl, af, (const double*)Y, (const double*)Wn, ldwn, nz,
                               lanczos_steps, rtol, maxit, nlml, grad, st);
  return with_timeout_check(pl, s, st);
}

agp_status agp_plan_landmarks(agp_plan pl, int n_landmarks, int32_t* idx, int cap, int* count,
                              void* stream) {
  if (!pl || !count || n_landmarks < 1 || n_landmarks > kMaxLandmarks || cap < 0 ||
      (cap > 0 && !idx))
    return set_error(AGP_EINVAL, "bad arguments (n_landmarks must be in [1, 480])");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> L;
  const agp_status s = pl->prec == AGP_F32 ? precond_landmarks<float>(pl, n_landmarks, L, st)
                                           : precond_landmarks<double>(pl, n_landmarks, L, st);
  if (s != AGP_OK) return s;
  *count = (int)L.size();
  if ((int)L.size() > cap) return set_error(AGP_EINVAL, "idx holds fewer entries than the landmark set");
  std::copy(L.begin(), L.end(), idx);
  return AGP_OK;
}

agp_status agp_nlml_grad_pc(agp_plan pl, const void* Y, const void* Wn, int64_t ldwn,
                            const double* Wk, int nz, int n_landmarks, int lanczos_steps,
                            double rtol, int maxit, double* nlml, double* grad, void* stream) {
  if (!pl || !Y || !Wn || !Wk || !nlml || !grad || nz < 1 || nz > 31 || ldwn < nz ||
      lanczos_steps < 1 || lanczos_steps > kMaxLanczos || (rtol > 0 && maxit < 1) || !(rtol >= 0))
    return set_error(AGP_EINVAL, "bad arguments");
  if (n_landmarks < 1 || n_landmarks > kMaxLandmarks)
    return set_error(AGP_EINVAL, "n_landmarks must be in [1, 480]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const agp_status s =
      pl->prec == AGP_F32
          ? nlml_pc_t<float>(pl, (const float*)Y, (const float*)Wn, ldwn, Wk, nz, n_landmarks,
                             lanczos_steps, rtol, maxit, nlml, grad, st)
          : nlml_pc_t<double>(pl, (const double*)Y, (const double*)Wn, ldwn, Wk, nz, n_landmarks,
                              lanczos_steps, rtol, maxit, nlml, grad, st);
  return with_timeout_check(pl, s, st);
}

agp_status agp_dot_columns(agp_plan pl, const void* A, int64_t lda, const void* B, int64_t ldb,
                           int R, double* out, void* stream) {
  if (!pl || !A || !B || !out || R < 1 || lda < R || ldb < R)
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* buf = nullptr;
  AGP_CUDA(cudaMallocAsync(&buf, sizeof(double) * (kMaxDotBlocks + 1) * R, st));
  agp_status s =
      pl->prec == AGP_F32
          ? col_dot((const float*)A, lda, (const float*)B, ldb, pl->n, R, buf,
                           buf + (int64_t)kMaxDotBlocks * R, st, pl)
          : col_dot((const double*)A, lda, (const double*)B, ldb, pl->n, R, buf,
                            buf + (int64_t)kMaxDotBlocks * R, st, pl);
  if (s == AGP_OK) {
    cudaError_t e = cudaMemcpyAsync(out, buf + (int64_t)kMaxDotBlocks * R, sizeof(double) * R,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    s = cuda_status(e, "agp_dot_columns");
  }
  cudaFreeAsync(buf, st);
  return with_timeout_check(pl, s, st);
}

agp_status agp_dot_columns_static(agp_prec prec, const void* A, int64_t lda, const void* B,
                                  int64_t ldb, int64_t n, int R, double* out, void* stream) {
  if (!A || !B || !out || n < 1 || lda < R || ldb < R)
    return set_error(AGP_EINVAL, "bad arguments");
  if (R < 1 || R > kStaticDotMaxR)
    return set_error(AGP_EINVAL, "agp_dot_columns_static: R must be in [1, 64]");
  if (prec != AGP_F32 && prec != AGP_F64) return set_error(AGP_EINVAL, "bad prec");
  double* scratch = nullptr;
  AGP_TRY(static_dot_scratch(&scratch));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = (int)std::min<int64_t>(kStaticDotBlocks, (n + kDotRows - 1) / kDotRows);
  const dim3 grid(nb, (R + 31) / 32);
  if (prec == AGP_F32)
    k_dot_partial<float, float><<<grid, kDotThreads, 0, st>>>((const float*)A, lda, (const float*)B,
                                                              ldb, n, R, scratch);
  else
    k_dot_partial<double, double><<<grid, kDotThreads, 0, st>>>((const double*)A, lda,
                                                                (const double*)B, ldb, n, R, scratch);
  k_dot_final<<<R, kDotFinalThreads, 0, st>>>(scratch, nb, R, out);
  return cuda_status(cudaGetLastError(), "agp_dot_columns_static");
}

agp_status agp_rademacher(agp_prec prec, int64_t n, int R, uint64_t seed, void* Z, int64_t ldz,
                          void* stream) {
  if (!Z || n < 1 || R < 1 || ldz < R || (prec != AGP_F32 && prec != AGP_F64))
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == AGP_F32)
    k_rademacher<float><<<nblk(n * R, 256), 256, 0, st>>>((float*)Z, ldz, n, R, seed);
  else
    k_rademacher<double><<<nblk(n * R, 256), 256, 0, st>>>((double*)Z, ldz, n, R, seed);
  return cuda_status(cudaGetLastError(), "agp_rademacher");
}

agp_status agp_nlml_grad_seed(agp_plan pl, const void* Y, int n_probes, int lanczos_steps,
                              uint64_t seed, double rtol, int maxit, double* nlml, double* grad,
                              void* stream) {
  if (!pl || !Y || n_probes < 1 || lanczos_steps < 1 || lanczos_steps > kMaxLanczos || !nlml ||
      !grad || !(rtol >= 0) || (rtol > 0 && maxit < 1))
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = pl->prec == AGP_F32 ? sizeof(float) : sizeof(double);
  void* Z = nullptr;
  AGP_CUDA(cudaMallocAsync(&Z, es * pl->n * n_probes, st));
  agp_status s = agp_rademacher(pl->prec, pl->n, n_probes, seed, Z, n_probes, stream);
  if (s == AGP_OK)
    s = pl->prec == AGP_F32
            ? nlml_t<float>(pl, (const float*)Y, (const float*)Z, n_probes, n_probes,
                            lanczos_steps, rtol, maxit, nlml, grad, st)
            : nlml_t<double>(pl, (const double*)Y, (const double*)Z, n_probes, n_probes,
                             lanczos_steps, rtol, maxit, nlml, grad, st);
  cudaFreeAsync(Z, st);
  return with_timeout_check(pl, s, st);
}

agp_status agp_nlml_grad(agp_plan pl, const void* Y, const void* Z, int64_t ldz, int nz,
                         int lanczos_steps, double rtol, int maxit, double* nlml, double* grad,
                         void* stream) {
  if (!pl || !Y || !Z || nz < 1 || ldz < nz || lanczos_steps < 1 ||
      lanczos_steps > kMaxLanczos || !nlml || !grad || (rtol > 0 && maxit < 1))
    return set_error(AGP_EINVAL, "bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const agp_status s =
      pl->prec == AGP_F32
          ? nlml_t<float>(pl, (const float*)Y, (const float*)Z, ldz, nz, lanczos_steps, rtol,
                          maxit, nlml, grad, st)
          : nlml_t<double>(pl, (const double*)Y, (const double*)Z, ldz, nz, lanczos_steps, rtol,
                           maxit, nlml, grad, st);
  return with_timeout_check(pl, s, st);
}

}  // extern "C"
