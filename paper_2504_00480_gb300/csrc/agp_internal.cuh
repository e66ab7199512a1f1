// Internal declarations of the GB300 additive-kernel fast summation library.
//
// Geometry of one feature window (Sec. 3.1 and Appendix A of the paper):
//   * d <= 3 coordinates per point, scaled into [-1/4, 1/4)^d.
//   * Bandwidth N (index set I_N = {-N/2..N/2-1}^d), oversampled grid of
//     n_os = 2N points per dimension at positions l / n_os.
//   * A point with u = x * n_os has base cell b = floor(u) in [-N/2, N/2) and
//     touches the 2s grid points l = b-s+1 .. b+s per dimension (Kaiser-Bessel
//     window of half-support s). Because |x| < 1/4 and s <= N/2 those grid
//     points never wrap around, and together they fill the "active box"
//     l in [lo, lo + W) with lo = -N/2 - s + 1 and W = N + 2s - 1. The grids
//     of this library store only that box: active index a = l - lo, and the
//     point's taps are a = c + t, c = b + N/2 (its cell), t = 0 .. 2s-1.
//   * Spectra keep k_1..k_{d-1} in [-N/2, N/2] (K = N+1 values) and the last
//     coordinate k_d in [0, N/2] (Kh = N/2+1 values, Hermitian half).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "agp.h"

namespace agp {

constexpr int kMaxDim = 3;
constexpr int kMaxWindows = 64;
constexpr int kItemPoints = 256;     // points per work item (one grid cell or part of one)
constexpr long long kDefaultWaitLimit = 1ll << 26;   // polls per bounded tensor-core wait

// Per-window view handed to the spreading / interpolation kernels.
template <typename T>
struct WinDev {
  const T* xs;            // sorted coordinates, [d][n]
  const int32_t* perm;    // sorted position -> caller's point index
  const T* wts;           // window values, sorted order, [n][window_wpp(d, s)]
  T* grid;                // active-box grid, [W^d][RC]
  const int32_t* cell_start;   // [cells + 1] first sorted point of every cell
  int64_t n;
  int N, n_os, W;
};

// Work units of the tensor-core kernels for d = 3 windows: runs of up to
// kRunCells consecutive cells along the last dimension (aligned to multiples
// of kRunCells, so one (t1, t2, t3) grid block of 2s + kRunCells - 1 planes
// covers all their points). int4 (window | L << 16, first cell, first sorted
// point, point count); L = 0 means a single cell (plain work items).
constexpr int kRunCells = 4;
// Points per run unit: longer runs are split into units of at most this many
// points (each a separate accumulation in tensor memory; the tensor cores'
// FP32 accumulation error grows with the number of MMAs summed into one
// accumulator).
constexpr int kRunPoints = 256;
// Outer boundary smoothing: largest order p, and the stride of one boundary
// polynomial record (2p coefficients, padded, then the constant kappa(1/2)).
constexpr int kBndMaxP = 8;
constexpr int kBndStride = 2 * kBndMaxP + 1;

// Window values stored per point and dimension: the 2s taps padded with zeros
// to a multiple of 4 (16-byte vector loads).
inline int window_ttp(int s) { return (2 * s + 3) / 4 * 4; }
// Window values stored per point: the first d-1 dimensions as window_ttp(s)
// values each (2s taps, zero padded), then the last dimension's 2s taps each
// written twice (v, v), so that packed FP32 pairs load them directly.
inline int window_wpp(int d, int s) { return (d - 1) * window_ttp(s) + 4 * s; }

// Per-window right-hand sides and outputs, used when the windows of one
// launch belong to different problems (batches): the kernels then take V,
// Out and the scale factors from this table instead of their arguments.
// scale multiplies the window's interpolated result.
template <typename T>
struct WinIO {
  const T* V;
  int64_t ldv;
  T* Out;
  int64_t ldo;
  T scale;
};

// Buffers of one window for the DFT stages (device table entry).
struct FftWin {
  void* grid;
  void* specA;
  void* specB;
  const void* tw;
  const void* dmul;
  const void* dmul_der;
};

// Windows with the same (d, N, s) processed by one launch per DFT stage.
struct FftGroup {
  int d = 0, N = 0, W = 0, count = 0;
  int64_t grid_elems = 0, dmul_elems = 0;
  FftWin* tab = nullptr;   // device [count]
};

// Kaiser-Bessel window of Appendix A in grid units, divided by I0(b s) so that
// its values are O(1) in FP32: psi(delta) = sinh(b r) / (pi I0(b s) r),
// r = sqrt(s^2 - delta^2), delta = x n_os - l in (-s, s]. `norm` = 1/(pi I0(b s)).
__device__ __forceinline__ float kb_psi(float delta, float s, float b, float norm) {
  float r2 = (s - delta) * (s + delta);
  if (r2 <= 0.f) return b * norm;
  float r = sqrtf(r2);
  return sinhf(b * r) / r * norm;
}
__device__ __forceinline__ double kb_psi(double delta, double s, double b, double norm) {
  double r2 = (s - delta) * (s + delta);
  if (r2 <= 0.0) return b * norm;
  double r = sqrt(r2);
  return sinh(b * r) / r * norm;
}

// kappa(r) (der = 0) or d kappa / d ell (der = 1) for the kernels of
// agp_kernel, from r^2, in FP64 (Sec. 2.1 eqs. (2.2)-(2.3), Sec. 4).
__device__ __forceinline__ double kernel_value(int kernel, double r2, double ell, int der) {
  if (kernel == AGP_GAUSS) {
    const double kv = exp(-r2 / (2.0 * ell * ell));
    return der ? kv * r2 / (ell * ell * ell) : kv;
  }
  if (kernel == AGP_MATERN12) {
    const double r = sqrt(r2);
    const double kv = exp(-r / ell);
    return der ? kv * r / (ell * ell) : kv;
  }
  if (kernel == AGP_MATERN32) {   // (1 + r/ell) e^{-r/ell}; derivative r^2/ell^3 e^{-r/ell}
    const double r = sqrt(r2);
    const double ex = exp(-r / ell);
    return der ? r2 / (ell * ell * ell) * ex : (1.0 + r / ell) * ex;
  }
  if (kernel == AGP_IMQ) {        // (1 + r^2/ell^2)^{-1/2}; derivative r^2/ell^3 (.)^{-3/2}
    const double q = 1.0 / (1.0 + r2 / (ell * ell));
    const double kv = sqrt(q);
    return der ? r2 / (ell * ell * ell) * kv * q : kv;
  }
  // sinc: sin(u)/u with u = r/ell; derivative (sin(u)/u - cos(u)) / ell, by its
  // series u^2/3 - u^4/30 + u^6/840 - u^8/45360 for u < 0.05 (cancellation)
  const double u = sqrt(r2) / ell;
  if (!der) return u < 1e-4 ? 1.0 - u * u / 6.0 : sin(u) / u;
  if (u < 0.05) {
    const double u2 = u * u;
    return u2 * (1.0 / 3 - u2 * (1.0 / 30 - u2 * (1.0 / 840 - u2 / 45360))) / ell;
  }
  return (sin(u) / u - cos(u)) / ell;
}

__device__ __forceinline__ float dev_floor(float x) { return floorf(x); }
__device__ __forceinline__ double dev_floor(double x) { return floor(x); }

// One coefficient job of a plan (a1): the kernel (der = 0) or ell-derivative
// (der = 1) coefficients of one window, computed in the scratch arrays s0/s1
// and left in b; dmul receives the spectral multipliers (plan precision).
struct CoefJob {
  double* s0 = nullptr;
  double* s1 = nullptr;
  double* b = nullptr;
  const double* costab = nullptr;
  const double* winhat = nullptr;
  void* dmul = nullptr;
  int N = 0, d = 0, der = 0;
  int64_t cells = 0, dmul_elems = 0;
};

// One window of a plan (host side).
struct Window {
  int d = 0, N = 0, n_os = 0, W = 0, K = 0, Kh = 0, s = 0;
  int feat[kMaxDim] = {0, 0, 0};
  int64_t cells = 0;         // N^d
  int64_t grid_elems = 0;    // W^d (per RHS column)
  int64_t spec_elems = 0;    // W^(d-1) * Kh (complex, per RHS column): max intermediate
  int64_t dmul_elems = 0;    // K^(d-1) * Kh
  // device buffers
  int32_t* perm = nullptr;       // [n]
  void* xs = nullptr;            // [d][n]
  void* wts = nullptr;           // [n][window_wpp(d, s)] Kaiser-Bessel values, sorted order
  double* costab = nullptr;      // [N][N] cos(2 pi l k / N) / N for the coefficient DFT
  int32_t* cell_start = nullptr; // [cells + 1]
  int4* items = nullptr;         // work items (window, cell, start, count)
  int64_t n_items = 0;
  double* b = nullptr;           // b_k on I_N^d (FP64)
  double* bder = nullptr;        // b_k of the ell-derivative kernel
  void* dmul = nullptr;          // spectral multiplier for K_s     [dmul_elems]
  void* dmul_der = nullptr;      // spectral multiplier for K_s^der [dmul_elems]
  void* winhat = nullptr;        // per-dim deconvolution n_os psi_hat(k), k in [-N/2, N/2] (prec)
  void* tw = nullptr;            // twiddles exp(-2 pi i k (a + lo) / n_os), [K][W] complex (prec)
  void* grid = nullptr;          // [grid_elems][rc_max] (prec)
  void* specA = nullptr;         // complex scratch [spec_elems][rc_max]
  void* specB = nullptr;
  std::vector<double> winhat_h;  // host copy of n_os psi_hat(k)
  FftWin* fft_self = nullptr;    // device table with this window alone
  FftGroup self_group() const {
    FftGroup g;
    g.d = d;
    g.N = N;
    g.W = W;
    g.count = 1;
    g.grid_elems = grid_elems;
    g.dmul_elems = dmul_elems;
    g.tab = fft_self;
    return g;
  }
};

}  // namespace agp

struct agp_plan_s {
  int64_t n = 0;
  int p = 0;
  int P = 0;
  int s = 0;
  int sigma_os = 2;
  agp_kernel kernel = AGP_GAUSS;
  agp_prec prec = AGP_F32;
  double ell = 1, sigma_f = 1, sigma_eps = 0;
  double kb_b = 0, kb_norm = 0;
  int rc_max = 32;
  int item_points = agp::kItemPoints;   // points per work item (bin size), see agp_plan_autotune
  int use_tc = 3;                // kernel family of spreading and interpolation (agp_plan_set_tensor_cores)
  double bnd_eps = 0.0;          // outer boundary smoothing of kappa_R: layer width (0: off)
  int bnd_p = 0;                 // ... and its order (derivatives matched at each end)
  double* bnd_poly = nullptr;    // [2][kBndStride] boundary polynomials (kernel, ell-derivative)
  agp::CoefJob* coef_jobs = nullptr;   // [2 P] coefficient jobs (device), see compute_coeffs
  double* coef_scratch = nullptr;      // their scratch arrays
  int n_coef_jobs = 0, coef_dmax = 0;
  int64_t coef_cells_max = 0, coef_dmul_max = 0;
  std::vector<agp::Window> win;
  void* wins_dev = nullptr;      // WinDev<T>[P]
  void* grid_maps = nullptr;     // FP32 plans with d = 3 windows: grid tensor maps [2][P] (RC 16, 32)
  int4* items_all = nullptr;     // work items of every window, grouped by d
  int4* runs3 = nullptr;         // tensor-core work units (cell runs) of the d = 3 windows
  int64_t n_runs3 = 0;
  int64_t items_by_d[agp::kMaxDim + 1] = {0, 0, 0, 0};   // offsets of each d group
  std::vector<agp::FftGroup> groups;   // windows grouped by (d, N) for the DFT stages
  int* err_dev = nullptr;        // device error flags
  // second stream for the d < 3 windows' spreading and interpolation while
  // the d = 3 launch runs (fork / join events), created with the plan
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  long long wait_limit = agp::kDefaultWaitLimit;   // polls per bounded mbarrier wait
  // stage profiler
  bool prof = false;
  struct Ev { int stage, dim; cudaEvent_t a, b; };
  std::vector<Ev> prof_ev;
  int64_t launches[4] = {0, 0, 0, 0};
};

namespace agp {

// ---- error plumbing (agp_plan.cu) ----
agp_status set_error(agp_status s, const std::string& msg);
agp_status cuda_status(cudaError_t e, const char* what);
// AGP_TIMEOUT (and the timeout bit cleared) if a bounded tensor-core wait of
// the plan expired since the last check, else AGP_OK. Synchronises `st`.
agp_status timeout_check(agp_plan_s* pl, cudaStream_t st);
// s, or AGP_TIMEOUT when s is a result (OK, NOT_CONVERGED, ENAN) and a wait
// expired meanwhile: for entry points that synchronise anyway.
agp_status with_timeout_check(agp_plan_s* pl, agp_status s, cudaStream_t st);

// ---- kernel launchers (agp_nufft.cu) ----
// Spread the columns V[:, 0..R) of the windows referenced by `items` (all of
// dimension d and cutoff s) onto their grids, which the caller has zeroed.
// RC = grid column count (32, 8, 1 for FP32; 4, 1 for FP64). With io !=
// nullptr every window takes its V and ldv from io[window] instead.
// Right-hand sides processed per pass of spreading / DFT / interpolation for
// R requested columns (the grid holds that many columns per point).
int rhs_block_width(agp_prec prec, int R);

template <typename T>
cudaError_t spread_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, const T* V, int64_t ldv, int R,
                         cudaStream_t st);
// Tensor-core spreading (agp_spread_tc.cu): FP32, d = 3, RC = 16 or 32, s = 4 or 5.
// err receives bit 2 if a bounded wait expired.
bool spread_tc_supported(int d, int s, int RC);
cudaError_t spread_items_tc(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                            int64_t n_items, int s, const float* V, int64_t ldv, int R, int rc,
                            int* err, long long spin, cudaStream_t st);
// Persistent warp-specialised tensor-core spreading with A in tensor memory
// (agp_spread_tm.cu): FP32, d = 3, RC = 16 or 32, s = 4 or 5 (V rows are
// staged 16 bytes at a time when 16-byte aligned, else 4); units are the cell
// runs of the plan. Each unit's accumulator block is added into the grid by
// one bulk tensor reduction through `grid_maps`, the window's grid tensor map
// for this RC (encode_grid_maps; n_win maps, those of the d = 3 windows set).
bool spread_tm_supported(int d, int s, int RC);
cudaError_t spread_units_tm(const WinDev<float>* wins, const void* grid_maps, int n_win,
                            const int4* units, int64_t n_units, int s, const float* V,
                            int64_t ldv, int R, int rc, int* err, long long spin,
                            cudaStream_t st);
// Tensor maps of the grids of a plan's d = 3 windows (FP32) for the
// spreading epilogue's bulk reductions: RC = 16 maps then RC = 32 maps, n_win
// each, written to `out` (host memory, 64-byte aligned, 2 n_win maps of 128
// bytes). Entries of other windows are zero. False if the driver's encoder is
// unavailable or refuses a map.
constexpr int kGridMapBytes = 128;
bool encode_grid_maps(const WinDev<float>* wins_host, const int* win_d, int n_win, int s,
                      void* out);
// Persistent warp-specialised tensor-core interpolation with A in tensor
// memory (agp_interp_tm.cu): FP32, d = 3, RC = 16 or 32, s = 4 or 5.
bool interp_tm_supported(int d, int s, int RC, int R);
cudaError_t interp_units_tm(const WinDev<float>* wins, int n_win, const int4* units,
                            int64_t n_units, int s, float* Out, int64_t ldo, int R, float scale, int rc, int* err,
                            long long spin, cudaStream_t st);
// spread_items, or spread_items_tc when `tc` is set and the case is supported
// (spin: polls per bounded wait of the tensor-core kernel)
template <typename T>
cudaError_t spread_items_sel(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                             int64_t n_items, int d, int s, int RC, const T* V, int64_t ldv, int R,
                             int tc, int* err, long long spin, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (tc && spread_tc_supported(d, s, RC))
      return spread_items_tc(wins, io, items, n_items, s, V, ldv, R, RC, err, spin, st);
  }
  return spread_items<T>(wins, io, items, n_items, d, s, RC, V, ldv, R, st);
}
// Tensor-core interpolation (agp_interp_tc.cu): FP32, d = 3, RC = 16 or 32, s = 4 or 5.
bool interp_tc_supported(int d, int s, int RC);
cudaError_t interp_items_tc(const WinDev<float>* wins, const WinIO<float>* io, const int4* items,
                            int64_t n_items, int s, float* Out, int64_t ldo, int R, float scale,
                            int rc, int* err, long long spin, cudaStream_t st);
// Interpolate the grids of those windows and add scale * result into
// Out[:, 0..R) (with io: Out, ldo and scale of io[window]).
template <typename T>
cudaError_t interp_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, T* Out, int64_t ldo, int R,
                         T scale, cudaStream_t st);

// interp_items, or interp_items_tc when `tc` is set and the case is supported
template <typename T>
cudaError_t interp_items_sel(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                             int64_t n_items, int d, int s, int RC, T* Out, int64_t ldo, int R,
                             T scale, int tc, int* err, long long spin, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (tc && interp_tc_supported(d, s, RC))
      return interp_items_tc(wins, io, items, n_items, s, Out, ldo, R, scale, RC, err, spin, st);
  }
  return interp_items<T>(wins, io, items, n_items, d, s, RC, Out, ldo, R, scale, st);
}

// ---- landmark (Nystrom) preconditioner (agp_precond.cu) ----
// M^{-1} = sigma_eps^{-2} (I - B Ginv B^T), B = K_{:,L} [n][k] stored in the
// plan precision, Ginv = (sigma_eps^2 K_LL + B^T B)^{-1} [k][k] in FP64. The
// products with B are accumulated to about FP64 accuracy in both precisions
// (FP32 plans: compensated FP32 arithmetic on hi/lo splits).
constexpr int kMaxLandmarks = 480;      // requested landmarks
constexpr int kMaxLandmarkSet = 512;    // after merging the windows' sets
struct Precond {
  int k = 0, rmax = 0, slices = 0;
  int64_t n = 0, rows_per_slice = 0;
  double inv_s2 = 0;
  void* B = nullptr;
  double* Ginv = nullptr;
  double* partial = nullptr;   // [slices][k][rmax]
  double* t1 = nullptr;        // [k][rmax]
  void* t2 = nullptr;          // FP64 plans: [k][rmax] double; FP32: hi, lo [2][k][rmax] float
  float* xsplit = nullptr;     // FP32 plans: hi, lo parts of the input [2][n][rmax]
  void* Bd = nullptr;          // dB/dell [n][k] (only with PrecondNlml)
};
// What the preconditioned likelihood needs besides M^{-1} (host FP64, k x k
// row-major): G^{-1}, K_LL^{-1}, the lower Cholesky factor of K_LL, the
// ell-derivative of K_LL and B^T dB/dell, and the log-determinants of G and K_LL.
struct PrecondNlml {
  std::vector<double> Ginv, K, Kinv, Kchol, Kder, BtBder;   // K includes delta I
  double logdet_G = 0.0, logdet_K = 0.0;
  double delta = 0.0;                                        // jitter on K_LL
};
void precond_free(Precond* pc);
template <typename T>
agp_status precond_build(agp_plan_s* pl, int k, int rmax, Precond* pc, cudaStream_t st,
                         PrecondNlml* ex = nullptr);
// out[j][r] = sum_i Bsel[i][j] X[i][r] (Bsel = B, or dB/dell when der), X FP64
// [n][R] with leading dimension R, out host [k][R]; accumulated like M^{-1}.
template <typename T>
agp_status precond_bt(const Precond& pc, int der, const double* X, int R, double* out,
                      cudaStream_t st);
// Z[i][r] = a W[i][r] + sum_j B[i][j] Tk[j][r] for r < nz: W in the plan
// precision [n][ldw], Tk device FP64 [k][nz], Z [n][ldz] in the plan precision.
template <typename T>
agp_status precond_affine(const Precond& pc, double a, const T* W, int64_t ldw, const double* Tk,
                          int nz, T* Z, int64_t ldz, cudaStream_t st);
// The landmark set the preconditioner uses for a request of k landmarks
// (sorted, no repeats; host vector).
template <typename T>
agp_status precond_landmarks(agp_plan_s* pl, int k, std::vector<int32_t>& out, cudaStream_t st);
// Y = M^{-1} X for X, Y FP64 [n][R] with leading dimension R (R <= 32).
template <typename T>
agp_status precond_apply(const Precond& pc, const double* X, double* Y, int R, cudaStream_t st);

// ---- additive AFN preconditioner (agp_afn.cu) ----
// M = Phi diag(K_LL, (G^T G)^{-1}) Phi^T with the landmark block factorised
// exactly and G the FSAI factor of the Schur complement (FP64 throughout).
constexpr int kAfnMaxFill = 128;
struct Afn {
  int64_t n = 0, m = 0, nnz = 0, rows_per_slice = 0;
  int k = 0, fill = 0, rmax = 0, slices = 0, kernel = 0;
  double ell = 0, sigma_f = 0, sigma_eps = 0;   // hyperparameters it was built for
  double logdet = 0;                            // log det M
  std::vector<int32_t> landmarks;               // host copy of L
  int32_t* L = nullptr;       // [k] landmark indices (ascending)
  int32_t* F = nullptr;       // [m] the other indices (ascending)
  double* Ci = nullptr;       // [k][k] C^{-1}, C the lower Cholesky factor of K_LL
  double* W = nullptr;        // [m][k] K_FL C^{-T}
  int32_t* J = nullptr;       // [m][fill] pattern positions, ascending, row's own last
  int32_t* len = nullptr;     // [m] entries per row
  double* Gval = nullptr;     // [m][fill]
  int32_t* colptr = nullptr;  // G^T: [m + 1]
  int32_t* colrow = nullptr;  // [nnz]
  double* colval = nullptr;   // [nnz]
  double *v = nullptr, *h = nullptr, *partial = nullptr;   // apply workspace
  double *t = nullptr, *u = nullptr, *w = nullptr;
  double* C = nullptr;        // [k][k] C (lower; zeros above the diagonal)
  // likelihood data (afn_build_derivs): derivatives with the landmarks and
  // the pattern held fixed, in the order ell, sigma_f, sigma_eps
  bool has_der = false;
  std::vector<double> KLL_h, C_h, Ci_h, dKLL_h;   // host [k][k]: K_LL, C, C^{-1}, dK_LL/dell
  double quad_sum[3] = {0, 0, 0};   // sum_t G_t^T dS[J_t, J_t] G_t
  double* Dl = nullptr;       // [m][k] (dK_FL/dell) C^{-T}
  double* dGval = nullptr;    // [3][m][fill] dG/dtheta on the pattern
  int32_t* lvl_rows = nullptr;        // rows of G ordered by level (triangular solve)
  std::vector<int64_t> lvl_off;       // host: level l holds lvl_rows[lvl_off[l] .. lvl_off[l+1])
};
void afn_free(Afn* af);
template <typename T>
agp_status afn_build(agp_plan_s* pl, int k, int fill, int rmax, Afn* af, cudaStream_t st);
// Y = M^{-1} X for FP64 blocks X [n][ldx], Y [n][ldy], R <= rmax columns.
agp_status afn_apply(const Afn& af, const double* X, int64_t ldx, double* Y, int64_t ldy, int R,
                     cudaStream_t st);
// Host copies of the landmarks [k] and the pattern [m][fill] (either may be null).
agp_status afn_pattern(const Afn& af, int32_t* landmarks, int32_t* J, cudaStream_t st);
// Derivative data for the likelihood gradient (once per object).
template <typename T>
agp_status afn_build_derivs(agp_plan_s* pl, Afn* af, cudaStream_t st);
// Y[t][r] = (G^{-1} X)[t][r] for FP64 [m][R] blocks (level-scheduled forward
// substitution; R <= 32).
agp_status afn_trsv(const Afn& af, const double* X, double* Y, int R, cudaStream_t st);
// Y = dG_theta X for FP64 [m][R] blocks (theta = 0, 1, 2).
agp_status afn_dg_apply(const Afn& af, int theta, const double* X, double* Y, int R,
                        cudaStream_t st);
// out[j][r] = sum_a A[a][j] X[a][r] over the m rows (A = W or Dl), host [k][R].
agp_status afn_wt(const Afn& af, const double* A, const double* X, int R, double* out,
                  cudaStream_t st);

// ---- DFT stages (agp_fft.cu), one launch per stage for a group of windows ----
template <typename T>
cudaError_t fft_forward(const FftGroup& g, int RC, cudaStream_t st);   // grid -> spectrum
template <typename T>
cudaError_t fft_inverse(const FftGroup& g, int RC, cudaStream_t st);   // spectrum -> grid
template <typename T>
cudaError_t spectral_multiply(const FftGroup& g, int der, int RC, cudaStream_t st);
template <typename T>
cudaError_t zero_grids(const FftGroup& g, int RC, cudaStream_t st);
// The whole DFT stage (forward, multiply, inverse) of groups with d = 2 or 3
// in three launches (agp_dft.cu); the spectrum is not kept.
bool dft_fused_supported(const FftGroup& g);
template <typename T>
cudaError_t dft_stage(const FftGroup* groups, int n_groups, int der, int RC, cudaStream_t st);

}  // namespace agp
