/*
 * agp.h -- C ABI of the GB300 additive-kernel NFFT fast summation library.
 *
 * Paper: "Preconditioned Additive Gaussian Processes with Fourier Acceleration"
 * (arXiv 2504.00480). The library applies the regularised additive kernel
 * matrix
 *
 *     K_hat = sigma_f^2 (K_1 + ... + K_P) + sigma_eps^2 I        (Sec. 2.1)
 *
 * and its hyperparameter derivatives to blocks of vectors. Each sub-kernel
 * K_s acts on the features of one window W_s (d_s <= 3) and is applied by the
 * NFFT-based fast summation of Sec. 3.1 eq. (3.3): Kaiser-Bessel spreading
 * onto an oversampled grid (adjoint NFFT), a d-dimensional DFT, a multiply by
 * the kernel's Fourier coefficients b_k (eq. (3.2)), an inverse DFT and
 * interpolation back to the points (NFFT), Appendix A. The output is the real
 * part of eq. (3.3).
 *
 * Conventions shared by every entry point
 *  - Precision: a plan is FP32 or FP64 (agp_prec); X, V, Out and every other
 *    floating-point device buffer of that plan have that element type.
 *  - Layout: point data are row-major [n][ld] (one row per point). Blocks of
 *    right-hand sides are RHS-minor: column r of V is V[i*ldv + r].
 *  - Ownership: the caller owns every buffer passed in and the CUDA stream;
 *    the plan owns its sorted copies of the points and all scratch. Device
 *    pointers are plain CUDA device addresses (e.g. a torch tensor's
 *    data_ptr()). `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - Asynchrony: compute calls only enqueue work on `stream` and return;
 *    calls that return host values (marked "synchronises") wait for it.
 *    A plan with windows of d = 3 and of d < 3 runs the latter's spreading
 *    and interpolation on a second stream of its own, forked from and
 *    joined back to `stream` by events inside the call, so the call still
 *    orders like a single launch on `stream` (and can be captured with it).
 *  - Errors: every call returns an agp_status; nothing is printed and nothing
 *    exits. agp_status_string() names a status; agp_last_error() gives the
 *    message of the last failing call on this thread.
 *  - Thread safety: calls on one plan must not overlap; distinct plans are
 *    independent.
 */
#ifndef AGP_H
#define AGP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct agp_plan_s* agp_plan;

typedef enum {
  AGP_OK = 0,
  AGP_EINVAL = 1,        /* invalid argument (sizes, pointers, unsupported combination) */
  AGP_EDOMAIN = 2,       /* a point of some window lies outside [-1/4, 1/4)^d (Sec. 3.1) */
  AGP_ECUDA = 3,         /* a CUDA runtime call failed */
  AGP_ENOMEM = 4,        /* device allocation failed */
  AGP_NOT_CONVERGED = 5, /* an iterative solve stopped at maxit above its tolerance */
  AGP_TIMEOUT = 6,       /* a bounded device wait expired */
  AGP_ENAN = 7           /* a non-finite value was met */
} agp_status;

/* Sec. 2.1 eq. (2.2): Gaussian exp(-r^2/(2 ell^2)), Matern(1/2) exp(-r/ell);
 * Matern(3/2) of the remark in Sec. 4, (1 + r/ell) exp(-r/ell) (its l = sqrt(3) ell);
 * two further kernels named in Sec. 4, normalised to 1 at r = 0 with c = ell:
 * the inverse multiquadric (1 + r^2/ell^2)^{-1/2} and sinc sin(r/ell) / (r/ell). */
typedef enum {
  AGP_GAUSS = 0,
  AGP_MATERN12 = 1,
  AGP_MATERN32 = 2,
  AGP_IMQ = 3,
  AGP_SINC = 4
} agp_kernel;
typedef enum { AGP_F32 = 0, AGP_F64 = 1 } agp_prec;
typedef enum { AGP_D_ELL = 0, AGP_D_SIGMA_F = 1, AGP_D_SIGMA_EPS = 2 } agp_param;

/* Plan description (Sec. 2.1 and Sec. 3.1).
 *  n, p, X, ldx : n points with p features, device [n][ldx], ldx >= p.
 *                 X may be freed after agp_plan_create returns.
 *  P, win_ptr, win_feat : feature windows W_1..W_P as a host CSR array:
 *                 window s uses features win_feat[win_ptr[s] .. win_ptr[s+1]-1]
 *                 (0-based, 1 <= d_s <= 3, windows disjoint).
 *  N            : host [P], Fourier bandwidth per window (the paper's m; the
 *                 index set is I_N = {-N/2..N/2-1}^d). N in {8, 16, 32, 64}.
 *  cutoff       : window half-support s in oversampled grid cells, 2 <= s <= 6
 *                 and s <= N/2 (Appendix A).
 *  sigma_os     : oversampling factor of the NFFT grid, must be 2 (grid of
 *                 n_os = 2N points per dimension).
 *  kernel, ell, sigma_f, sigma_eps : kernel and hyperparameters (ell > 0).
 *  prec         : element type of every floating-point buffer of the plan.
 * Every point of every window must lie in [-1/4, 1/4)^{d_s} (Sec. 3.1 scales
 * the data there); otherwise agp_plan_create returns AGP_EDOMAIN. */
typedef struct {
  int64_t n;
  int p;
  const void* X;
  int64_t ldx;
  int P;
  const int* win_ptr;
  const int* win_feat;
  const int* N;
  int cutoff;
  int sigma_os;
  agp_kernel kernel;
  double ell, sigma_f, sigma_eps;
  agp_prec prec;
} agp_plan_desc;

/* Build a plan: sort every window's points into grid cells (cell index
 * floor(x * n_os) per coordinate, exact for the power-of-two n_os), copy the
 * sorted coordinates, and compute the Fourier coefficients b_k of the kernel
 * and of its ell-derivative (Sec. 3.1 eq. (3.2), Sec. 3.2 eq. (3.4)) with the
 * Kaiser-Bessel deconvolution factors (Appendix A). Synchronises `stream`.
 * On success *out owns device memory until agp_plan_destroy. */
agp_status agp_plan_create(agp_plan* out, const agp_plan_desc* desc, void* stream);

/* Release the plan and all its device memory. Synchronises the device. */
agp_status agp_plan_destroy(agp_plan plan);

/* New hyperparameters (ell > 0, sigma_f, sigma_eps). Recomputes b_k for the
 * kernel and its ell-derivative on `stream` (Sec. 3.1 eq. (3.2)); asynchronous. */
agp_status agp_set_hyper(agp_plan plan, double ell, double sigma_f, double sigma_eps,
                         void* stream);

/* Out = K_hat V (add_noise = 1) or sigma_f^2 sum_s K_s V (add_noise = 0), with
 * each K_s applied by the fast summation of Sec. 3.1 eq. (3.3) (real part).
 * V: device [n][ldv], columns 0..R-1 used; Out: device [n][ldo]; R >= 1;
 * ldv, ldo >= R. Out must not overlap V. Asynchronous on `stream`. */
agp_status agp_matvec(agp_plan plan, const void* V, int64_t ldv, void* Out, int64_t ldo,
                      int R, int add_noise, void* stream);

/* Out = (dK_hat / dtheta) V for theta = ell (sigma_f^2 sum_s K_s^der, Sec. 2.1
 * eq. (2.3), applied with the derivative-kernel coefficients of Sec. 3.2
 * eq. (3.4)), sigma_f (2 sigma_f sum_s K_s) or sigma_eps (2 sigma_eps I).
 * Arguments as agp_matvec. Asynchronous on `stream`. */
agp_status agp_deriv_matvec(agp_plan plan, agp_param which, const void* V, int64_t ldv,
                            void* Out, int64_t ldo, int R, void* stream);

/* ---- Spectra and the spectral quadratic form (Sec. 3.2) -----------------------
 * For the gradient of a scalar L = sum_r G_r^T K_hat V_r with respect to the
 * hyperparameters, eq. (3.4) moves the ell-derivative onto the Fourier
 * coefficients, so G^T (dK/dell) V needs only the adjoint sums of G and V:
 *   G^T K_s V      = sum_k D_k Re(conj(g_k) v_k),
 *   G^T K_s^der V  = sum_k D^der_k Re(conj(g_k) v_k),
 * where g_k, v_k are the forward DFTs of the spread grids of G and V and D,
 * D^der the spectral multipliers (b_k over the squared window transform,
 * Appendix A) of the kernel and of its ell-derivative -- exactly the
 * operator agp_matvec applies, since interpolation is the transpose of
 * spreading. No interpolation and no second spread are needed.
 *
 * agp_spectra_size: number of complex elements (plan precision) of the
 * spectra of R columns (all windows). */
agp_status agp_spectra_size(agp_plan plan, int R, int64_t* elems);

/* Out = K_hat V as agp_matvec, and the forward spectra of V (all windows,
 * R columns) written to spec: device, agp_spectra_size(R) complex elements
 * of the plan precision, an internal layout that only agp_spectral_form
 * reads. With Out = NULL only the spectra are computed (spreading and the
 * forward DFT). Asynchronous on `stream`. */
agp_status agp_matvec_spectra(agp_plan plan, const void* V, int64_t ldv, void* Out, int64_t ldo,
                              int R, int add_noise, void* spec, void* stream);

/* out[r] = G_r^T Op V_r from the spectra A (of G) and B (of V) of
 * agp_matvec_spectra, for Op = sigma_f^2 sum_s K_s (which = -1), the
 * ell-derivative sigma_f^2 sum_s K_s^der (which = AGP_D_ELL, Sec. 3.2 eq.
 * (3.4)) or 2 sigma_f sum_s K_s (which = AGP_D_SIGMA_F), with the plan's
 * current coefficients. out: device double[R], overwritten (FP64
 * accumulation). Asynchronous on `stream`. */
agp_status agp_spectral_form(agp_plan plan, int which, const void* A, const void* B, int R,
                             double* out, void* stream);

/* Adjoint NFFT of one window (Appendix A, the inner sum of eq. (3.3)):
 * chat[r][k] ~= sum_j V[j][r] exp(-2 pi i k . x_j^{W_s}), k in I_N^d, stored
 * row-major over (k_1 + N/2, ..., k_d + N/2), as interleaved (re, im) pairs.
 * chat: device [R][N^d][2]. Asynchronous on `stream`. */
agp_status agp_adjoint_nfft(agp_plan plan, int window, const void* V, int64_t ldv, int R,
                            void* chat, void* stream);

/* Real part of the NFFT of one window (Appendix A, the outer sum of
 * eq. (3.3)): Out[i][r] = Re sum_{k in I_N^d} fhat[r][k] exp(2 pi i k . x_i).
 * fhat: device [R][N^d][2] laid out as agp_adjoint_nfft's output; Out:
 * device [n][ldo] (overwritten). Asynchronous on `stream`. */
agp_status agp_nfft_real(agp_plan plan, int window, const void* fhat, int R, void* Out,
                         int64_t ldo, void* stream);

/* Grid-cell index floor(x_t * n_os) of every point in one window, in the
 * caller's point order: bins: device int32 [n][d]. Asynchronous. */
agp_status agp_plan_bins(agp_plan plan, int window, int32_t* bins, void* stream);

/* Fourier coefficients b_k (deriv = 0) or those of the ell-derivative kernel
 * (deriv = 1) of one window for the current ell, as computed on the device:
 * b: host double [N^d], row-major over (k_1 + N/2, ..., k_d + N/2).
 * Synchronises `stream`. */
agp_status agp_plan_coeffs(agp_plan plan, int window, int deriv, double* b, void* stream);

/* Work items ("bins"): the points of each window are sorted by grid cell and
 * cut into work items of at most `points` points of one cell (default 256);
 * one work item is one CTA of spreading and interpolation. Rebuilds the work
 * items (16 <= points <= 4096, else AGP_EINVAL). Batches created on the plan
 * before the call keep the old items: create them again. Synchronises
 * `stream`. (Not from the paper: a property of the GPU layout.) */
agp_status agp_plan_set_item_points(agp_plan plan, int points, void* stream);

/* Autotuner: times `reps` applications of K_hat to R columns (device
 * scratch allocated and freed here, CUDA events on `stream`) first for each
 * kernel family of agp_plan_set_tensor_cores (FP32 plans: 1, 2, 3 and 0) at
 * the current work-item size, then, with the fastest family, for each
 * work-item size in {64, 128, 256, 512, 1024}, and keeps the fastest pair.
 * Results are cached for the process, keyed by precision, cutoff, pass
 * width, R, the windows' (d, N) and floor(log2 n): a later plan with the
 * same key takes the cached choice without timing. points, ms: optional host
 * outputs, the chosen size and its mean time per call in milliseconds
 * (agp_plan_tensor_cores gives the chosen family). Batches must be created
 * after this call. Synchronises `stream`. (Not from the paper: a property of
 * the GPU layout.) */
agp_status agp_plan_autotune(agp_plan plan, int R, int reps, int* points, double* ms,
                             void* stream);

/* The plan's kernel family (the value of agp_plan_set_tensor_cores). */
agp_status agp_plan_tensor_cores(agp_plan plan, int* mode);

/* Which kernels run the d = 3 spreading and interpolation of the first pass
 * of an R-column application (V or Out rows with stride ldv >= R; the
 * kernels take any stride and alignment): 3 the persistent tensor-memory
 * kernel over cell runs, 2 the shared-memory tensor-core kernel over cell
 * runs, 1 the tensor-core kernel over work items, 0 the FMA kernel; -1 when
 * the plan has no d = 3 window. Depends on the plan's precision, cutoff,
 * kernel family (agp_plan_set_tensor_cores) and on R; a family-3 plan takes
 * family 2 for an interpolation pass whose second 16-column half would be
 * empty (R <= RC - 16). The persistent spreading kernel adds each unit's
 * block into the grid by one bulk tensor reduction through tensor maps of
 * the plan's grids, encoded at plan creation with the driver's
 * cuTensorMapEncodeTiled; if the driver offers no encoder or refuses a map,
 * the plan's spreading reports and runs family 2 instead. */
agp_status agp_plan_kernel_families(agp_plan plan, int R, int64_t ldv, int* spread, int* interp);

/* Forget every cached autotuner result of the process. */
agp_status agp_autotune_clear_cache(void);

/* Size queries: n, number of windows, and the number of work items (point
 * chunks) of one window. */
agp_status agp_plan_query(agp_plan plan, int64_t* n, int* P, int window, int* d,
                          int* N, int64_t* n_items);

/* Batched conjugate gradients for K_hat X = B (Sec. 1: CG with zero initial
 * guess, one independent recursion per column; the iterates x, r, p in FP64,
 * the matvec in the plan precision, every scalar -- column dot products,
 * alpha, beta, residual norms -- in FP64 on the device). Residual
 * replacement: every 5 iterations, a column whose recursive residual has
 * fallen 10x since its last recomputation, or has reached rtol, gets
 * r = b - K_hat x recomputed (x split into its plan-precision rounding and
 * the remainder, two matvecs), so that the recursion cannot drift from the
 * operator's true residual. Column r stops when its relative residual
 * |b - K_hat x|_2 / |b|_2, so recomputed, is <= rtol, or after maxit
 * iterations (relres then holds the last recursive value).
 * B: device [n][ldb]; Xsol: device [n][ldx], overwritten with the iterates;
 * iters, relres: optional host arrays [R] (NULL to skip).
 * n_landmarks: 0 for plain CG, or 1..480 for CG preconditioned with the
 * landmark part of the paper's additive AFN preconditioner (Sec. 2.3):
 * ceil(n_landmarks / P) landmarks per feature window by farthest point
 * sampling (first landmark: point 0; ties: lowest index), merged, and
 * M = K_{:,L} (K_LL + delta I)^{-1} K_{L,:} + sigma_eps^2 I (exact kernel;
 * delta starts at 1e-6 sigma_f^2 P and grows 100-fold, at most four times,
 * while the FP64 Cholesky of G = sigma_eps^2 (K_LL + delta I) + B^T B,
 * B = K_{:,L}, meets a non-positive pivot, which happens when the landmarks
 * outnumber the kernel's numerical rank) applied by the Woodbury identity with
 * an FP64 Cholesky factor; needs sigma_eps > 0 and R <= 32. The stopping test stays on the unpreconditioned residual.
 * Returns AGP_NOT_CONVERGED if some column stopped above rtol (Xsol holds the
 * last iterate). Synchronises `stream`. */
agp_status agp_pcg_solve(agp_plan plan, const void* B, int64_t ldb, void* Xsol, int64_t ldx,
                         int R, double rtol, int maxit, int n_landmarks, int* iters,
                         double* relres, void* stream);

/* The landmark set that agp_pcg_solve uses for the same n_landmarks
 * (1..480; Sec. 2.3): ceil(n_landmarks / P) indices per feature window by
 * farthest point sampling on that window's coordinates (in the plan
 * precision; first landmark point 0; each next one maximises the squared
 * Euclidean distance to those already chosen, evaluated and compared in
 * FP64, ties to the lowest index), merged into increasing order without
 * repeats.
 * idx: host int32 array with room for cap entries; count: host int, set to
 * the size of the set (at most P * ceil(n_landmarks / P)). Returns AGP_EINVAL
 * if cap is smaller (count is still set). Synchronises `stream`. */
agp_status agp_plan_landmarks(agp_plan plan, int n_landmarks, int32_t* idx, int cap, int* count,
                              void* stream);

/* Spreading and interpolation on the tensor cores (FP32 plans, d = 3
 * windows, s = 4 or 5, passes of 9 to 16 right-hand sides on 16-column grids
 * and of 17 or more on 32-column grids; other cases keep the FP32 FMA
 * path). Per work item, spreading's update of the cell's
 * (2s)^2 x (2s R) grid block is the matrix product [(t1, t2) x points] x
 * [points x (t3, r)] of window-value matrices, and interpolation's sum over
 * the first two dimensions is the product [points x (t1, t2)] x
 * [(t1, t2) x (t3, r)] with the grid block; both run as tcgen05.mma on TF32
 * operands split into a rounded part and its remainder, of which the tensor
 * cores use the TF32 bits (three products, about FP32 accuracy), accumulated
 * in FP32.
 * enable: 3 (the default for FP32 plans) both persistent warp-specialised
 * kernels with the A operand in tensor memory -- the fastest family
 * measured (interpolation needs R > RC - 16, else its pass runs on the
 * shared-memory kernel); 1 spreading by the persistent kernel,
 * interpolation by the kernel with both operands in shared memory; 2 both
 * kernels with operands in shared memory; 0 off (FMA path only). */
agp_status agp_plan_set_tensor_cores(agp_plan plan, int enable);

/* Outer boundary smoothing of the periodic kernel kappa_R (Sec. 3.1: the
 * periodic extension may be smoothed at its outer boundary; the paper's own
 * runs leave it unsmoothed, which is this library's default). With
 * eps_b > 0 and p > 0, kappa_R(r) is kappa(r) for r <= a = 1/2 - eps_b, on
 * the layer a < r < 1/2 the two-point Taylor polynomial T of degree 2p - 1
 * with T^(j)(a) = kappa^(j)(a) and T(1/2) = kappa(1/2), T^(j)(1/2) = 0
 * (1 <= j < p), and kappa(1/2) for r >= 1/2; its periodic continuation is
 * p - 1 times continuously differentiable, so the truncated Fourier series
 * of eq. (3.1) converges faster for smooth kernels. The ell-derivative
 * kernel of eq. (3.4) is regularised the same way. kappa_R equals kappa at
 * every point difference only if |x_i - x_j| <= 1/2 - eps_b, so every
 * window's scaled points must lie in the ball |x| <= 1/4 - eps_b/2.
 * eps_b: layer width in [0, 1/4]; p: order in [0, 8] (eps_b = 0 or p = 0
 * switches the smoothing off). Recomputes the Fourier coefficients on
 * `stream` (and again at every agp_set_hyper with a new ell).
 * Returns AGP_EINVAL for arguments out of range and AGP_EDOMAIN if a point
 * lies outside the ball (the plan then keeps its previous setting).
 * Synchronises `stream`. */
agp_status agp_plan_set_boundary(agp_plan plan, double eps_b, int p, void* stream);

/* AGP_TIMEOUT if a bounded wait inside a tensor-core kernel expired since
 * the last check (the flag is then cleared), else AGP_OK. Synchronises
 * `stream`. The entry points that synchronise anyway (agp_pcg_solve,
 * agp_pcg_solve_afn, agp_nlml_grad, agp_nlml_grad_pc, agp_nlml_grad_afn,
 * agp_dot_columns) make this check themselves and return AGP_TIMEOUT in
 * place of their result status; after asynchronous calls (agp_matvec,
 * agp_deriv_matvec, agp_batch_matvec) call it before trusting the output.
 * A batch reports through the error word of its first plan. */
agp_status agp_plan_check(agp_plan plan, void* stream);

/* Number of polls after which a bounded mbarrier wait inside the plan's
 * tensor-core kernels gives up (0: the default, 2^26). On expiry the CTA
 * agrees on the failure, stops issuing tensor-core work, drains what it
 * issued (with the default bound), records AGP_TIMEOUT for agp_plan_check
 * and leaves its part of the output unwritten, so the result is invalid but
 * the device stays usable. A small limit is only useful to exercise that
 * path. (Not from the paper: a property of the GPU kernels.) */
agp_status agp_plan_set_wait_limit(agp_plan plan, int64_t polls);

/* Negative log marginal likelihood and its gradient with respect to
 * (ell, sigma_f, sigma_eps), estimated as in Sec. 1 eqs. (1.4) and (1.5) with
 * M = I:
 *   nlml    = 1/2 (y^T alpha + (1/nz) sum_i z_i^T logm(K_hat) z_i + n log 2 pi)
 *   grad[j] = 1/2 (-alpha^T dK_j alpha + (1/nz) sum_i u_i^T dK_j z_i)
 * One batched CG run on [y, z_1..z_nz]: every probe column runs
 * lanczos_steps iterations (its CG coefficients give the Lanczos matrix of
 * stochastic Lanczos quadrature; u_i is its CG iterate); the y column runs
 * lanczos_steps iterations too when rtol = 0, else to relative residual rtol
 * (at most maxit iterations) -- alpha is its iterate. A column whose
 * relative residual falls to 1e-12 (FP64 plans) or 1e-6 (FP32 plans) stops
 * there and its Lanczos matrix ends at that step: its Krylov space is then
 * invariant to working precision, the quadrature exact to that level, and
 * further steps would be set by rounding noise (Lanczos breakdown). The
 * preconditioned variants apply the same rule.
 * Y: device [n]; Z: device [n][ldz], nz >= 1 probe columns (e.g. Rademacher,
 * drawn by the caller); 1 <= lanczos_steps <= 64. nlml: host double; grad:
 * host double[3] (ell, sigma_f, sigma_eps). Synchronises `stream`. */
agp_status agp_nlml_grad(agp_plan plan, const void* Y, const void* Z, int64_t ldz, int nz,
                         int lanczos_steps, double rtol, int maxit, double* nlml, double* grad,
                         void* stream);

/* agp_nlml_grad with n_probes Rademacher probes drawn on the device from
 * `seed` (agp_rademacher), the form of the estimate that Sec. 1 describes;
 * every argument as in agp_nlml_grad. Allocates the n x n_probes probe
 * block on `stream` for the call. Synchronises `stream`. */
agp_status agp_nlml_grad_seed(agp_plan plan, const void* Y, int n_probes, int lanczos_steps,
                              uint64_t seed, double rtol, int maxit, double* nlml, double* grad,
                              void* stream);

/* Rademacher probe block for Hutchinson's trace estimator (Sec. 1): entry
 * Z[i*ldz + c] (i < n, c < R) is +1 when the top bit of output i R + c of the
 * counter-based SplitMix64 generator started at `seed` is 0, else -1
 * (Steele, Lea and Flood, OOPSLA 2014: output j mixes the state
 * seed + (j + 1) 0x9E3779B97F4A7C15). Z: device, element type `prec`.
 * Asynchronous on `stream`. (The generator is not from the paper, which
 * leaves the probes' source open.) */
agp_status agp_rademacher(agp_prec prec, int64_t n, int R, uint64_t seed, void* Z, int64_t ldz,
                          void* stream);

/* The same estimate with the landmark preconditioner M = B K_LL^{-1} B^T +
 * sigma_eps^2 I of agp_pcg_solve (Sec. 2.3), as in Sec. 1 eqs. (1.3)-(1.5):
 *   nlml    = 1/2 (y^T alpha + log det M + (1/nz) sum_i q_i + n log 2 pi)
 *   grad[j] = 1/2 (-alpha^T dK_j alpha + tr(M^{-1} dM_j)
 *                  + (1/nz) sum_i (u_i^T dK_j p_i - p_i^T dM_j p_i))
 * log det M and tr(M^{-1} dM_j) are exact (FP64, through the k x k Cholesky
 * factors); the probes z_i = sigma_eps wn_i + B C^{-T} wk_i (C C^T = K_LL)
 * have covariance M for caller-drawn vectors w_i = [wn_i; wk_i] with
 * covariance I; q_i is the SLQ estimate of z~_i^T logm(M^{-1/2} K_hat
 * M^{-1/2}) z~_i, z~_i = M^{-1/2} z_i, from exactly lanczos_steps PCG steps
 * on K_hat x = z_i (u_i is the iterate, p_i = M^{-1} z_i). The y column runs
 * lanczos_steps PCG steps when rtol = 0, else to relative residual rtol (at
 * most maxit steps).
 * Y: device [n]; Wn: device [n][ldwn] in the plan precision, 1 <= nz <= 31
 * columns; Wk: host double [k][nz] with k the size of the landmark set for
 * n_landmarks (agp_plan_landmarks); 1 <= n_landmarks <= 480; needs
 * sigma_eps > 0. nlml: host double; grad: host double[3] (ell, sigma_f,
 * sigma_eps). Returns AGP_ENAN (gradient still written) when SLQ meets a
 * non-positive Ritz value or K_LL is not positive definite. Synchronises
 * `stream`. */
agp_status agp_nlml_grad_pc(agp_plan plan, const void* Y, const void* Wn, int64_t ldwn,
                            const double* Wk, int nz, int n_landmarks, int lanczos_steps,
                            double rtol, int maxit, double* nlml, double* grad, void* stream);

/* ---- Additive AFN preconditioner (Sec. 2.3) ----------------------------------
 * The adaptive factorised Nystrom preconditioner for additive kernels: the
 * landmark block of K_hat is factorised exactly and the Schur complement of
 * the remaining points is approximated by a factorised sparse approximate
 * inverse (FSAI) with at most `fill` entries per row. With the landmarks L
 * first and the other points F (increasing index) after them,
 *   S = K_FF - K_FL K_LL^{-1} K_LF     (blocks of K_hat, noise included),
 *   M = Phi diag(K_LL, (G^T G)^{-1}) Phi^T,   Phi = [I 0; K_FL K_LL^{-1} I],
 * with the exact kernel in FP64. G is lower triangular: row t (the t-th point
 * of F) holds t and its min(fill - 1, t) nearest earlier points of F, by the
 * squared Euclidean distance over all window features (in window order)
 * computed in FP64, ties to the lower index; on that pattern J_t,
 * G[t, J_t] = g / sqrt(g_t)
 * with S[J_t, J_t] g = e_t. M's landmark rows equal those of K_hat; with a
 * full pattern M = K_hat; with fill = 1 G is the inverse square root of S's
 * diagonal. log det M = log det K_LL - 2 sum_t log G_tt.
 * The landmark count is the caller's (the paper's adaptive rank estimate is
 * not made). The object keeps the hyperparameters of the plan at creation;
 * build a new one after agp_set_hyper. Memory: about (12 fill + 8 k) bytes per
 * point plus 24 * 32 bytes per point of apply workspace. */
typedef struct agp_afn_s* agp_afn;

/* Build M for the plan's current hyperparameters. n_landmarks: 1..480,
 * landmarks chosen as in agp_pcg_solve (agp_plan_landmarks); fill: 1..128.
 * Needs sigma_eps > 0. Returns AGP_ENAN if a factorisation meets a
 * non-positive pivot (*out stays NULL). Synchronises `stream`. */
agp_status agp_afn_create(agp_afn* out, agp_plan plan, int n_landmarks, int fill, void* stream);
agp_status agp_afn_destroy(agp_afn afn);
/* Y = M^{-1} V for FP64 device blocks V [n][ldv] and Y [n][ldy] (row-major,
 * 1 <= R <= 32 columns; Y must not alias V). Asynchronous on `stream`. */
agp_status agp_afn_apply(agp_afn afn, const double* V, int64_t ldv, double* Y, int64_t ldy, int R,
                         void* stream);
/* Size of the landmark set, nonzeros of G and log det M (each may be NULL). */
agp_status agp_afn_info(agp_afn afn, int* n_landmarks, int64_t* nnz, double* logdet);
/* Host copies of the landmark indices (int32 [k]) and the pattern (int32
 * [n - k][fill]: positions in F, increasing, the row's own position last,
 * -1 after). Either pointer may be NULL. Synchronises `stream`. */
agp_status agp_afn_pattern(agp_afn afn, int32_t* landmarks, int32_t* J, void* stream);
/* Preconditioned CG on K_hat Xsol = B with the AFN preconditioner, as
 * agp_pcg_solve otherwise (R <= 32; stopping test on the unpreconditioned
 * relative residual). AGP_EINVAL if `afn` was built for other hyperparameters
 * or another point count. Synchronises `stream`. */
agp_status agp_pcg_solve_afn(agp_plan plan, agp_afn afn, const void* B, int64_t ldb, void* Xsol,
                             int64_t ldx, int R, double rtol, int maxit, int* iters,
                             double* relres, void* stream);

/* NLML estimate and gradient with the AFN preconditioner M of `afn` (Sec. 1
 * eqs. (1.3)-(1.5)), the estimator of agp_nlml_grad_pc with
 *   probes     z_i = Phi [C wL_i; G^{-1} wF_i] (covariance M), where wL_i and
 *              wF_i are the landmark rows and the other rows of column i of Wn;
 *   log det M  = log det K_LL - 2 sum_t log G_tt;
 *   tr(M^{-1} dM_j) = d log det M / dtheta_j (exact, with the landmarks and
 *              the pattern of G held fixed);
 *   p_i^T dM_j p_i from the exact derivative of M (dG row by row).
 * G^{-1} is applied by forward substitution level by level (the rows of a
 * level depend only on earlier levels). The first call builds the
 * derivative data of `afn` (about 3 fill + k doubles per point).
 * Y: device [n]; Wn: device [n][ldwn] in the plan precision, 1 <= nz <= 31
 * columns with covariance I; 1 <= lanczos_steps <= 64; rtol / maxit as in
 * agp_nlml_grad_pc. nlml: host double; grad: host double[3] (ell, sigma_f,
 * sigma_eps). AGP_EINVAL if `afn` was built for other hyperparameters.
 * Synchronises `stream`. */
agp_status agp_nlml_grad_afn(agp_plan plan, agp_afn afn, const void* Y, const void* Wn,
                             int64_t ldwn, int nz, int lanczos_steps, double rtol, int maxit,
                             double* nlml, double* grad, void* stream);

/* ---- Batches of independent problems ----------------------------------------
 * Many independent GP problems of different sizes (independent plans, each
 * with its own points, windows and hyperparameters) applied together: every
 * stage of the matvec runs as ONE launch over the work items of all problems
 * (the spread and interpolation kernels take each window's vectors from a
 * device table), so the per-problem launch overhead disappears and small
 * problems fill the GPU together. All plans must have the same precision and
 * cutoff; the batch refers to them, so they must outlive it. */
typedef struct agp_batch_s* agp_batch;

/* All plans must share precision, cutoff and the tensor-core setting
 * (agp_plan_set_tensor_cores); AGP_EINVAL otherwise. The batch's tensor-core
 * kernels use the wait limit and the error word of plans[0]. */
agp_status agp_batch_create(agp_batch* out, const agp_plan* plans, int nprob, void* stream);
agp_status agp_batch_destroy(agp_batch batch);

/* Bind the right-hand sides and outputs: problem q uses V[q] (device
 * [n_q][ldv[q]]) and Out[q] (device [n_q][ldo[q]], must not overlap V[q]),
 * columns 0..R-1, 1 <= R <= 32 (FP32 plans) or R <= 4 (FP64 plans). V, ldv,
 * Out, ldo are host arrays [nprob]. Reads every plan's current sigma_f and
 * sigma_eps: bind again after agp_set_hyper changes them (a new ell needs no
 * rebinding). Synchronises `stream`. */
agp_status agp_batch_bind(agp_batch batch, const void* const* V, const int64_t* ldv,
                          void* const* Out, const int64_t* ldo, int R, void* stream);

/* For every bound problem q: Out_q = K_hat_q V_q (which = -1) or
 * Out_q = (dK_hat_q / dtheta) V_q (which = an agp_param), as agp_matvec and
 * agp_deriv_matvec. Enqueues a fixed sequence of kernels (no allocation, no
 * host synchronisation), so it can be captured in a CUDA graph once it has
 * run outside capture. */
agp_status agp_batch_matvec(agp_batch batch, int which, void* stream);

/* Column dot products out[r] = sum_i A[i][r] * B[i][r], r < R, accumulated in
 * FP64 (two-pass, deterministic order) for blocks of the plan precision.
 * A: device [n][lda], B: device [n][ldb], n = the plan's point count;
 * out: host double[R]. Synchronises `stream`; returns AGP_TIMEOUT if a
 * tensor-core wait of the plan expired before (see agp_plan_check). */
agp_status agp_dot_columns(agp_plan plan, const void* A, int64_t lda, const void* B, int64_t ldb,
                           int R, double* out, void* stream);

/* Column dot products like agp_dot_columns, for callers that may not allocate
 * device memory: code that runs where cudaMalloc / cudaMallocAsync are not
 * allowed or not wanted -- inside a framework or memory pool that owns all of
 * the device's memory, or in a latency-critical loop that must not trigger an
 * allocation (and the synchronisation or pool growth that can come with it).
 * The paper has no counterpart: this is a property of the library, not of
 * the method.
 *  - Allocates nothing: the partial sums live in a fixed device array of the
 *    library (512 blocks x 64 columns of doubles, 256 KB), held by every GPU
 *    that loads the library until the process exits. Nothing in it needs to
 *    start at zero: each call writes every partial sum it reads.
 *  - The first call on a device looks the array up for that device (with it
 *    current) and caches the address per device index; make that first call
 *    before any stream capture. The cached address is not valid after the
 *    device is reset (cudaDeviceReset) within the same process: do not call
 *    this entry point after such a reset.
 *  - Every call shares the array: calls whose work overlaps on the GPU (two
 *    streams, or two threads) race. Serialise them.
 *  - prec: element type of A and B. A: device [n][lda], B: device [n][ldb];
 *    out: device double[R], written with sum_i A[i][r] * B[i][r] (FP64).
 *    R must be 1..64 (AGP_EINVAL otherwise). Asynchronous on `stream`. */
agp_status agp_dot_columns_static(agp_prec prec, const void* A, int64_t lda, const void* B,
                                  int64_t ldb, int64_t n, int R, double* out, void* stream);

/* Stage profiler (tracing). When enabled, the library records a pair of CUDA
 * events on the caller's stream around every kernel launch of the matvec
 * path, per stage: 0 = spreading, 1 = DFT + spectral multiply, 2 =
 * interpolation, 3 = other (output init, solver vector kernels).
 * agp_profile_read (synchronises `stream`) returns, per stage, the summed
 * device time in milliseconds and the number of kernel launches since the
 * last reset, and resets when reset != 0. Launch counts are kept even when
 * timing is disabled. */
typedef struct {
  double ms[4];                /* device time per stage */
  int64_t launches[4];         /* kernel launches per stage */
  double ms_by_dim[4][4];      /* spreading / interpolation time per window dimension d = 1..3 */
  int64_t timed_by_dim[4][4];  /* number of launches behind ms_by_dim[stage][d] */
} agp_profile_t;

agp_status agp_profile_enable(agp_plan plan, int enable);
agp_status agp_profile_read(agp_plan plan, agp_profile_t* out, int reset, void* stream);

/* Name of a status code (static string). */
const char* agp_status_string(agp_status s);

/* Message of the last failing call on the calling thread (static storage). */
const char* agp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AGP_H */
