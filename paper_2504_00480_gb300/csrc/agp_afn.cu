// Additive AFN preconditioner (Sec. 2.3): the landmark block of K_hat is
// factorised exactly, the Schur complement of the remaining points gets a
// factorised sparse approximate inverse (FSAI) with a fixed fill level.
//
// With the landmarks L (farthest point sampling per window, merged) first
// and the remaining points F (ascending index) after them,
//     K_hat = [K_LL K_LF; K_FL K_FF]   (noise sigma_eps^2 on every diagonal),
//     S = K_FF - K_FL K_LL^{-1} K_LF   (Schur complement, m = n - k rows),
//     M = Phi diag(K_LL, (G^T G)^{-1}) Phi^T,  Phi = [I 0; K_FL K_LL^{-1} I],
// where G is lower triangular with at most `fill` entries per row: row t
// holds t and its fill-1 nearest earlier positions u < t of F (squared
// Euclidean distance over the window features in FP64, the squared
// differences summed in feature order; ties to the lower position), and
// G[t, J_t] = g / sqrt(g_t) with S[J_t, J_t] g = e_t, so that
// G S G^T has unit diagonal. With C the lower Cholesky factor of K_LL and
// W = K_FL C^{-T} ([m][k]),
//     M^{-1} r:  v = C^{-1} r_L;  t = r_F - W v;  w = G^T G t;
//                out_F = w;  out_L = C^{-T} (v - W^T w),
//     log det M = log det K_LL - 2 sum_t log G_tt.
// Everything is FP64: the exact kernel entries, S[J, J] and its Cholesky
// factor (one CTA per row of G, in shared memory), and the apply's vectors.
//
// Device layout: J and Gval [m][fill] (row-major, positions ascending with
// t last, -1 / 0 padding), and G^T as compressed columns (colptr [m + 1],
// colrow, colval) filled once at build time so that the apply gathers
// instead of scattering.
#include <algorithm>
#include <cmath>
#include <vector>

#include "agp_exact.cuh"

namespace agp {
namespace {

constexpr int kKnnWarps = 8;
constexpr unsigned kFull = 0xFFFFFFFFu;

// shared memory of one warp of k_knn_lower: kAfnMaxFill distances (FP64) and
// positions, then the row's pf features (FP64); a multiple of 8 bytes
__host__ __device__ constexpr size_t knn_warp_bytes(int pf) {
  return (size_t)kAfnMaxFill * (sizeof(double) + sizeof(int)) + (size_t)pf * sizeof(double);
}

// out[a][j] = sf2 d kernel_sum(rows_a, L_j) / dell, FP64 [m][k]
template <typename T>
__global__ void k_kernel_cols_rows(const WinPts<T>* __restrict__ wp, int P, int64_t n,
                                   const int32_t* __restrict__ rows, int64_t m,
                                   const int32_t* __restrict__ lm, int k, int kernel, double ell,
                                   double sf2, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t a = e / k;
  const int j = (int)(e - a * k);
  out[e] = sf2 * kernel_sum<T>(wp, P, n, rows[a], lm[j], kernel, ell, 1);
}

// out[a][j] = sf2 kernel_sum(rows_a, L_j), FP64 [m][k]
template <typename T>
__global__ void k_kernel_rows(const WinPts<T>* __restrict__ wp, int P, int64_t n,
                              const int32_t* __restrict__ rows, int64_t m,
                              const int32_t* __restrict__ lm, int k, int kernel, double ell,
                              double sf2, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t a = e / k;
  const int j = (int)(e - a * k);
  out[e] = sf2 * kernel_sum<T>(wp, P, n, rows[a], lm[j], kernel, ell, 0);
}

// out = the lower triangle of A (k x k), zeros above the diagonal
__global__ void k_lower_copy(const double* __restrict__ A, int k, double* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int i = (int)(e / k), j = (int)(e - (int64_t)i * k);
  out[e] = j <= i ? A[e] : 0.0;
}

// W[a][j] = sum_{i <= j} Ci[j][i] Bf[a][i]   (W = Bf C^{-T}, Ci = C^{-1} lower)
__global__ void k_times_lower_t(const double* __restrict__ Bf, int64_t m, int k,
                                const double* __restrict__ Ci, double* __restrict__ W) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t a = e / k;
  const int j = (int)(e - a * k);
  double s = 0.0;
  for (int i = 0; i <= j; ++i) s = fma(Ci[(int64_t)j * k + i], Bf[a * k + i], s);
  W[e] = s;
}

// xf[c0 + t][a] = coordinate t of point F_a in FP64 (one window, caller order [d][n])
template <typename T>
__global__ void k_gather_feat(const T* __restrict__ x, int d, int64_t n,
                              const int32_t* __restrict__ F, int64_t m, int c0,
                              double* __restrict__ xf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * d) return;
  const int t = (int)(e / m);
  const int64_t a = e - (int64_t)t * m;
  xf[(int64_t)(c0 + t) * m + a] = (double)x[(int64_t)t * n + F[a]];
}

// Pattern of row a (one warp per row): the fill-1 nearest earlier positions
// kept in a list sorted by (distance, position) in shared memory; candidates
// u = 0 .. a-1 are scanned 32 at a time and inserted one by one. Writes
// J[a][0 .. len) ascending with a last, -1 after, and len[a].
__global__ void __launch_bounds__(kKnnWarps * 32)
k_knn_lower(const double* __restrict__ xf, int pf, int64_t m, int fill, int32_t* __restrict__ J,
            int32_t* __restrict__ len) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t a = (int64_t)blockIdx.x * kKnnWarps + warp;
  if (a >= m) return;   // the whole warp leaves together
  // per warp: the sorted list's distances and positions, then the row's features
  double* ld = reinterpret_cast<double*>(smem_raw + (size_t)warp * knn_warp_bytes(pf));
  int* lp = reinterpret_cast<int*>(ld + kAfnMaxFill);
  double* q = reinterpret_cast<double*>(lp + kAfnMaxFill);
  for (int c = lane; c < pf; c += 32) q[c] = xf[(int64_t)c * m + a];
  __syncwarp();
  const int cap = fill - 1;
  int cnt = 0;
  double thr_d = 0.0;
  int thr_p = 0;
  for (int64_t u0 = 0; u0 < a && cap > 0; u0 += 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < a;
    double dist = 0.0;
    if (valid)
      for (int c = 0; c < pf; ++c) {
        const double dd = xf[(int64_t)c * m + u] - q[c];
        dist = __dadd_rn(dist, __dmul_rn(dd, dd));
      }
    const bool pass =
        valid && (cnt < cap || dist < thr_d || (dist == thr_d && (int)u < thr_p));
    unsigned mask = __ballot_sync(kFull, pass);
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const double dc = __shfl_sync(kFull, dist, src);
      const int uc = (int)(u0 + src);
      if (cnt == cap && !(dc < thr_d || (dc == thr_d && uc < thr_p))) continue;
      int below = 0;
      for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        const bool lt = e < cnt && (ld[e] < dc || (ld[e] == dc && lp[e] < uc));
        below += __popc(__ballot_sync(kFull, lt));
      }
      const int newcnt = min(cnt + 1, cap);
      double rd[kAfnMaxFill / 32];
      int rp[kAfnMaxFill / 32];
#pragma unroll
      for (int qq = 0; qq < kAfnMaxFill / 32; ++qq) {
        const int e = lane + 32 * qq;
        if (e > below && e < newcnt) {
          rd[qq] = ld[e - 1];
          rp[qq] = lp[e - 1];
        }
      }
      __syncwarp();
#pragma unroll
      for (int qq = 0; qq < kAfnMaxFill / 32; ++qq) {
        const int e = lane + 32 * qq;
        if (e > below && e < newcnt) {
          ld[e] = rd[qq];
          lp[e] = rp[qq];
        }
      }
      if (lane == 0) {
        ld[below] = dc;
        lp[below] = uc;
      }
      __syncwarp();
      cnt = newcnt;
      if (cnt == cap) {
        thr_d = ld[cap - 1];
        thr_p = lp[cap - 1];
      }
    }
  }
  // ascending positions: the rank of each entry among the chosen positions
  int32_t* row = J + a * fill;
  for (int e = lane; e < cnt; e += 32) {
    const int pe = lp[e];
    int rank = 0;
    for (int f = 0; f < cnt; ++f) rank += lp[f] < pe;
    row[rank] = pe;
  }
  for (int e = cnt + lane; e < fill; e += 32) row[e] = e == cnt ? (int32_t)a : -1;
  if (lane == 0) len[a] = cnt + 1;
}

// Row a of G (one CTA): S[J, J] in shared memory (lower triangle, stride
// fill + 1), its Cholesky factor R in place, then R^T g = e_last by columns.
// With DER, also the derivatives of the row for theta = (ell, sigma_f,
// sigma_eps) with the pattern fixed: v = dS[J, J] g, y = S[J, J]^{-1} v by
// two triangular solves with R, dG[a][J] = -y + g (g^T v) / 2 and
// quad[theta][a] = g^T v. With omega = sum_b g_b W_b, delta = sum_b g_b Dl_b
// (rows of W = K_FL C^{-T} and Dl = dK_FL/dell C^{-T} at the pattern),
// E = C^{-1} dK_LL/dell C^{-T} and Pm = C^{-1} C^{-T}:
//   v_ell[a]   = sum_b dK_ab g_b - Dl_a.omega - W_a.delta + W_a.(E omega)
//   v_sf[a]    = (2 / sigma_f) ([a = last] / g_last - s2 g_a - s2 W_a.(Pm omega))
//   v_seps[a]  = 2 sigma_eps (g_a + W_a.(Pm omega)),
// using S[J, J] g = e_last / g_last.
template <typename T, bool DER>
__global__ void __launch_bounds__(256)
k_fsai_rows(const WinPts<T>* __restrict__ wp, int P, int64_t n, const int32_t* __restrict__ F,
            const double* __restrict__ W, int k, const int32_t* __restrict__ J,
            const int32_t* __restrict__ len, int64_t m, int fill, int kernel, double ell,
            double sf, double se, double* __restrict__ Gval, double* __restrict__ logdiag,
            int* __restrict__ flag, const double* __restrict__ Dl, const double* __restrict__ E,
            const double* __restrict__ Pm, double* __restrict__ dGval, double* __restrict__ quad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* S = reinterpret_cast<double*>(smem_raw);
  __shared__ int pos[kAfnMaxFill], idx[kAfnMaxFill];
  __shared__ double acc[kAfnMaxFill], g[kAfnMaxFill];
  const int tid = threadIdx.x, bs = blockDim.x;
  const int64_t a = blockIdx.x;
  const int L = len[a];
  const int ldS = fill + 1;
  const double sf2 = sf * sf, s2 = se * se;
  for (int q = tid; q < L; q += bs) {
    pos[q] = J[a * fill + q];
    idx[q] = F[pos[q]];
    acc[q] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < L * L; e += bs) {
    const int i = e / L, j = e - i * L;
    if (j > i) continue;
    const double* wi = W + (int64_t)pos[i] * k;
    const double* wj = W + (int64_t)pos[j] * k;
    double c = 0.0;
    for (int q = 0; q < k; ++q) c = fma(wi[q], wj[q], c);
    S[i * ldS + j] = sf2 * kernel_sum<T>(wp, P, n, idx[i], idx[j], kernel, ell, 0) +
                     (i == j ? s2 : 0.0) - c;
  }
  __syncthreads();
  for (int j = 0; j < L; ++j) {
    const double piv = S[j * ldS + j];
    if (!(piv > 0.0)) {   // the same value for every thread: all leave together
      if (tid == 0) atomicExch(flag, 1);
      return;
    }
    const double rj = sqrt(piv);
    __syncthreads();
    for (int i = j + 1 + tid; i < L; i += bs) S[i * ldS + j] /= rj;
    if (tid == 0) S[j * ldS + j] = rj;
    __syncthreads();
    const int mm = L - j - 1;
    for (int e = tid; e < mm * mm; e += bs) {
      const int ii = j + 1 + e / mm, ll = j + 1 + e % mm;
      if (ll <= ii) S[ii * ldS + ll] -= S[ii * ldS + j] * S[ll * ldS + j];
    }
    __syncthreads();
  }
  for (int i = L - 1; i >= 0; --i) {
    if (tid == 0) g[i] = ((i == L - 1 ? 1.0 : 0.0) - acc[i]) / S[i * ldS + i];
    __syncthreads();
    for (int j = tid; j < i; j += bs) acc[j] = fma(S[i * ldS + j], g[i], acc[j]);
    __syncthreads();
  }
  for (int q = tid; q < fill; q += bs) Gval[a * fill + q] = q < L ? g[q] : 0.0;
  if (tid == 0) logdiag[a] = log(g[L - 1]);
  if constexpr (DER) {
    __shared__ double om[kMaxLandmarkSet], de[kMaxLandmarkSet], eom[kMaxLandmarkSet],
        pom[kMaxLandmarkSet];
    __shared__ double v[3][kAfnMaxFill], z[3][kAfnMaxFill], y[3][kAfnMaxFill],
        acc3[3][kAfnMaxFill];
    __shared__ double qd[3];
    for (int j = tid; j < k; j += bs) {
      double o = 0.0, d = 0.0;
      for (int b = 0; b < L; ++b) {
        o = fma(g[b], W[(int64_t)pos[b] * k + j], o);
        d = fma(g[b], Dl[(int64_t)pos[b] * k + j], d);
      }
      om[j] = o;
      de[j] = d;
    }
    __syncthreads();
    for (int j = tid; j < k; j += bs) {
      double e1 = 0.0, p1 = 0.0;
      for (int i = 0; i < k; ++i) {
        e1 = fma(E[(int64_t)j * k + i], om[i], e1);
        p1 = fma(Pm[(int64_t)j * k + i], om[i], p1);
      }
      eom[j] = e1;
      pom[j] = p1;
    }
    __syncthreads();
    for (int q = tid; q < L; q += bs) {
      const double* wa = W + (int64_t)pos[q] * k;
      const double* da = Dl + (int64_t)pos[q] * k;
      double s_dw = 0.0, s_wd = 0.0, s_we = 0.0, s_wp = 0.0;
      for (int j = 0; j < k; ++j) {
        s_dw = fma(da[j], om[j], s_dw);
        s_wd = fma(wa[j], de[j], s_wd);
        s_we = fma(wa[j], eom[j], s_we);
        s_wp = fma(wa[j], pom[j], s_wp);
      }
      double dkg = 0.0;
      for (int b = 0; b < L; ++b)
        dkg = fma(sf2 * kernel_sum<T>(wp, P, n, idx[q], idx[b], kernel, ell, 1), g[b], dkg);
      v[0][q] = dkg - s_dw - s_wd + s_we;
      v[1][q] = (2.0 / sf) * ((q == L - 1 ? 1.0 / g[L - 1] : 0.0) - s2 * g[q] - s2 * s_wp);
      v[2][q] = 2.0 * se * (g[q] + s_wp);
      acc3[0][q] = acc3[1][q] = acc3[2][q] = 0.0;
    }
    __syncthreads();
    // R z = v (forward, by columns)
    for (int i = 0; i < L; ++i) {
      if (tid < 3) z[tid][i] = (v[tid][i] - acc3[tid][i]) / S[i * ldS + i];
      __syncthreads();
      const int r = L - i - 1;
      for (int e = tid; e < 3 * r; e += bs) {
        const int th = e / r, j = i + 1 + e % r;
        acc3[th][j] = fma(S[j * ldS + i], z[th][i], acc3[th][j]);
      }
      __syncthreads();
    }
    for (int e = tid; e < 3 * L; e += bs) acc3[e / L][e % L] = 0.0;
    __syncthreads();
    // R^T y = z (backward, by columns)
    for (int i = L - 1; i >= 0; --i) {
      if (tid < 3) y[tid][i] = (z[tid][i] - acc3[tid][i]) / S[i * ldS + i];
      __syncthreads();
      for (int e = tid; e < 3 * i; e += bs) {
        const int th = e / i, j = e % i;
        acc3[th][j] = fma(S[i * ldS + j], y[th][i], acc3[th][j]);
      }
      __syncthreads();
    }
    if (tid < 3) {
      double q = 0.0;
      for (int b = 0; b < L; ++b) q = fma(g[b], v[tid][b], q);
      qd[tid] = q;
      quad[(int64_t)tid * m + a] = q;
    }
    __syncthreads();
    for (int e = tid; e < 3 * fill; e += bs) {
      const int th = e / fill, q = e - th * fill;
      dGval[((int64_t)th * m + a) * fill + q] = q < L ? fma(0.5 * qd[th], g[q], -y[th][q]) : 0.0;
    }
  }
}

__global__ void k_col_count(const int32_t* __restrict__ J, const int32_t* __restrict__ len,
                            int64_t m, int fill, int32_t* __restrict__ cnt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * fill) return;
  const int64_t a = e / fill;
  if ((int)(e - a * fill) < len[a]) atomicAdd(cnt + J[e], 1);
}

// exclusive prefix sum of in[0 .. m) into out[0 .. m], one CTA
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ in,
                                               int32_t* __restrict__ out, int64_t m) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (m + 1023) / 1024;
  const int64_t lo = tid * per, hi = min(m, lo + per);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += in[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (int q = 0; q < 1024; ++q) {
      const int64_t v = part[q];
      part[q] = run;
      run += v;
    }
    out[m] = (int32_t)run;
  }
  __syncthreads();
  int64_t run = part[tid];
  for (int64_t i = lo; i < hi; ++i) {
    out[i] = (int32_t)run;
    run += in[i];
  }
}

__global__ void k_col_fill(const int32_t* __restrict__ J, const int32_t* __restrict__ len,
                           const double* __restrict__ Gval, int64_t m, int fill,
                           const int32_t* __restrict__ colptr, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ colrow, double* __restrict__ colval) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * fill) return;
  const int64_t a = e / fill;
  if ((int)(e - a * fill) >= len[a]) return;
  const int v = J[e];
  const int slot = colptr[v] + atomicAdd(cursor + v, 1);
  colrow[slot] = (int32_t)a;
  colval[slot] = Gval[e];
}

// ---- apply ----

// v[j][r] = sum_{i <= j} Ci[j][i] X[L_i][r]
__global__ void k_afn_lm_in(const double* __restrict__ X, int64_t ldx,
                            const int32_t* __restrict__ L, int k, int R,
                            const double* __restrict__ Ci, double* __restrict__ v) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * R) return;
  const int j = e / R, r = e - j * R;
  double s = 0.0;
  for (int i = 0; i <= j; ++i) s = fma(Ci[(int64_t)j * k + i], X[(int64_t)L[i] * ldx + r], s);
  v[e] = s;
}

// t[a][r] = X[F_a][r] - sum_j W[a][j] v[j][r]: a warp per row, lanes = columns,
// v staged in shared memory
__global__ void __launch_bounds__(256)
k_afn_schur_in(const double* __restrict__ X, int64_t ldx, const int32_t* __restrict__ F,
               int64_t m, const double* __restrict__ W, int k, int R,
               const double* __restrict__ v, double* __restrict__ t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sv = reinterpret_cast<double*>(smem_raw);
  for (int e = threadIdx.x; e < k * R; e += blockDim.x) sv[e] = v[e];
  __syncthreads();
  const int lane = threadIdx.x % 32;
  if (lane >= R) return;
  for (int64_t a = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; a < m; a += (int64_t)gridDim.x * 8) {
    const double* wr = W + a * k;
    double s = X[(int64_t)F[a] * ldx + lane];
    for (int j = 0; j < k; ++j) s = fma(-wr[j], sv[j * R + lane], s);
    t[a * R + lane] = s;
  }
}

// u[a][r] = sum_q G[a][q] t[J[a][q]][r]: a warp per row
__global__ void __launch_bounds__(256)
k_afn_g(const double* __restrict__ Gval, const int32_t* __restrict__ J,
        const int32_t* __restrict__ len, int fill, int64_t m, int R, const double* __restrict__ t,
        double* __restrict__ u) {
  const int lane = threadIdx.x % 32;
  if (lane >= R) return;
  for (int64_t a = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; a < m; a += (int64_t)gridDim.x * 8) {
    const int L = len[a];
    double s = 0.0;
    for (int q = 0; q < L; ++q)
      s = fma(Gval[a * fill + q], t[(int64_t)J[a * fill + q] * R + lane], s);
    u[a * R + lane] = s;
  }
}

// w[a][r] = sum over column a of G of G[b][a] u[b][r]; also Y[F_a][r] = w
__global__ void __launch_bounds__(256)
k_afn_gt(const int32_t* __restrict__ colptr, const int32_t* __restrict__ colrow,
         const double* __restrict__ colval, int64_t m, int R, const double* __restrict__ u,
         double* __restrict__ w, const int32_t* __restrict__ F, double* __restrict__ Y,
         int64_t ldy) {
  const int lane = threadIdx.x % 32;
  if (lane >= R) return;
  for (int64_t a = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; a < m; a += (int64_t)gridDim.x * 8) {
    double s = 0.0;
    for (int e = colptr[a]; e < colptr[a + 1]; ++e)
      s = fma(colval[e], u[(int64_t)colrow[e] * R + lane], s);
    w[a * R + lane] = s;
    Y[(int64_t)F[a] * ldy + lane] = s;
  }
}

// partial[z][j][r] = sum over the rows a of slice z of W[a][j] w[a][r]
__global__ void __launch_bounds__(256)
k_afn_wt(const double* __restrict__ W, const double* __restrict__ w, int64_t m, int k, int R,
         int64_t rows_per_slice, double* __restrict__ partial) {
  const int r = threadIdx.x % 32;
  const int j0 = blockIdx.x * 32 + (threadIdx.x / 32) * 4;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_slice;
  const int64_t r1 = min(m, r0 + rows_per_slice);
  if (r >= R) return;
  int nq = k - j0;
  nq = nq < 0 ? 0 : (nq > 4 ? 4 : nq);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t a = r0; a < r1; ++a) {
    const double x = w[a * R + r];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) acc[q] = fma(W[a * k + j0 + q], x, acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < nq) partial[((int64_t)blockIdx.y * k + j0 + q) * R + r] = acc[q];
}

// h[i][r] = v[i][r] - sum_z partial[z][i][r]
__global__ void k_afn_lm_mid(const double* __restrict__ partial, int nz,
                             const double* __restrict__ v, int k, int R, double* __restrict__ h) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * R) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += partial[(int64_t)z * k * R + e];
  h[e] = v[e] - s;
}

// Y[L_j][r] = sum_{i >= j} Ci[i][j] h[i][r]
__global__ void k_afn_lm_out(const double* __restrict__ h, const int32_t* __restrict__ L, int k,
                             int R, const double* __restrict__ Ci, double* __restrict__ Y,
                             int64_t ldy) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * R) return;
  const int j = e / R, r = e - j * R;
  double s = 0.0;
  for (int i = j; i < k; ++i) s = fma(Ci[(int64_t)i * k + j], h[(int64_t)i * R + r], s);
  Y[(int64_t)L[j] * ldy + r] = s;
}

// One level of the forward substitution G y = x: for the rows t of the level
// (their dependencies are in earlier levels), y[t][r] = (x[t][r] -
// sum_{q < len - 1} G[t][q] y[J[t][q]][r]) / G[t][len - 1]. A warp per row.
__global__ void __launch_bounds__(256)
k_afn_trsv_level(const int32_t* __restrict__ rows, int64_t nrows, const double* __restrict__ Gval,
                 const int32_t* __restrict__ J, const int32_t* __restrict__ len, int fill, int R,
                 const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x % 32;
  if (lane >= R) return;
  for (int64_t q0 = (int64_t)blockIdx.x * 8 + threadIdx.x / 32; q0 < nrows;
       q0 += (int64_t)gridDim.x * 8) {
    const int64_t t = rows[q0];
    const int L = len[t];
    double s = x[t * R + lane];
    for (int q = 0; q < L - 1; ++q)
      s = fma(-Gval[t * fill + q], y[(int64_t)J[t * fill + q] * R + lane], s);
    y[t * R + lane] = s / Gval[t * fill + L - 1];
  }
}

// out[j][r] = sum_z partial[z][j][r]
__global__ void k_sum_slices(const double* __restrict__ partial, int nz, int k, int R,
                             double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * R) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += partial[(int64_t)z * k * R + e];
  out[e] = s;
}

inline int fsai_threads(int fill) { return fill <= 32 ? 64 : (fill <= 64 ? 128 : 256); }

}  // namespace

void afn_free(Afn* af) {
  if (!af) return;
  for (void* p : {(void*)af->L, (void*)af->F, (void*)af->Ci, (void*)af->W, (void*)af->J,
                  (void*)af->len, (void*)af->Gval, (void*)af->colptr, (void*)af->colrow,
                  (void*)af->colval, (void*)af->v, (void*)af->t, (void*)af->u, (void*)af->w,
                  (void*)af->partial, (void*)af->h, (void*)af->C, (void*)af->Dl,
                  (void*)af->dGval, (void*)af->lvl_rows})
    cudaFree(p);
  *af = Afn();
}

template <typename T>
agp_status afn_build(agp_plan_s* pl, int k_req, int fill, int rmax, Afn* af, cudaStream_t st) {
  const int64_t n = pl->n;
  const int P = pl->P;
  if (!(pl->sigma_eps > 0)) return set_error(AGP_EINVAL, "the AFN preconditioner needs sigma_eps > 0");
  if (fill < 1 || fill > kAfnMaxFill) return set_error(AGP_EINVAL, "AFN fill must be in 1..128");
  if (k_req < 1 || k_req > kMaxLandmarks)
    return set_error(AGP_EINVAL, "AFN landmarks must be in 1..480");
  if (rmax < 1 || rmax > 32) return set_error(AGP_EINVAL, "AFN: 1..32 right-hand sides");
  CallerPoints<T> cp;
  AGP_TRY(caller_points<T>(pl, cp, st));
  std::vector<int32_t> lms;
  AGP_TRY(select_landmarks<T>(pl, cp, k_req, lms, st));
  const int k = (int)lms.size();
  if (k > kMaxLandmarkSet) return set_error(AGP_EINVAL, "AFN: more than 512 landmarks after merging");
  std::vector<int32_t> fh;
  fh.reserve(n - k);
  {
    size_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (q < lms.size() && lms[q] == i) {
        ++q;
        continue;
      }
      fh.push_back((int32_t)i);
    }
  }
  const int64_t m = (int64_t)fh.size();
  af->n = n;
  af->m = m;
  af->k = k;
  af->fill = fill;
  af->rmax = rmax;
  af->ell = pl->ell;
  af->sigma_f = pl->sigma_f;
  af->sigma_eps = pl->sigma_eps;
  af->kernel = pl->kernel;
  af->landmarks = lms;
  const double sf2 = pl->sigma_f * pl->sigma_f;
  const double s2 = pl->sigma_eps * pl->sigma_eps;
  WinPts<T>* wpd = nullptr;
  AGP_CUDA(cudaMallocAsync(&wpd, sizeof(WinPts<T>) * P, st));
  AGP_CUDA(cudaMemcpyAsync(wpd, cp.wp.data(), sizeof(WinPts<T>) * P, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMalloc(&af->L, sizeof(int32_t) * k));
  AGP_CUDA(cudaMemcpyAsync(af->L, lms.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
  // K_LL (noise included) -> C -> Ci = C^{-1}, log det K_LL
  double *KLL = nullptr, *dg = nullptr;
  int* flag = nullptr;
  AGP_CUDA(cudaMallocAsync(&KLL, sizeof(double) * k * k, st));
  AGP_CUDA(cudaMallocAsync(&dg, sizeof(double) * k, st));
  AGP_CUDA(cudaMallocAsync(&flag, sizeof(int), st));
  AGP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  AGP_CUDA(cudaMalloc(&af->Ci, sizeof(double) * k * k));
  k_kernel_block<T><<<nblk((int64_t)k * k, 256), 256, 0, st>>>(wpd, P, n, af->L, k, pl->kernel,
                                                               pl->ell, sf2, 0, s2, KLL);
  k_cholesky<<<1, 1024, 0, st>>>(KLL, k, flag);
  k_tri_inverse<<<nblk(k, 128), 128, 0, st>>>(KLL, k, af->Ci);
  AGP_CUDA(cudaMalloc(&af->C, sizeof(double) * k * k));
  k_lower_copy<<<nblk((int64_t)k * k, 256), 256, 0, st>>>(KLL, k, af->C);
  k_diag<<<nblk(k, 128), 128, 0, st>>>(KLL, k, dg);
  std::vector<double> diag(k);
  int hflag = 0;
  AGP_CUDA(cudaGetLastError());
  AGP_CUDA(cudaMemcpyAsync(diag.data(), dg, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(KLL, st);
  cudaFreeAsync(dg, st);
  if (hflag) {
    cudaFreeAsync(flag, st);
    cudaFreeAsync(wpd, st);
    return set_error(AGP_ENAN, "AFN: the landmark block is not positive definite");
  }
  double logdet = 0.0;
  for (int j = 0; j < k; ++j) logdet += 2.0 * std::log(diag[j]);
  if (m > 0) {
    AGP_CUDA(cudaMalloc(&af->F, sizeof(int32_t) * m));
    AGP_CUDA(cudaMemcpyAsync(af->F, fh.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    // W = K_FL C^{-T}
    double* Bf = nullptr;
    AGP_CUDA(cudaMallocAsync(&Bf, sizeof(double) * m * k, st));
    AGP_CUDA(cudaMalloc(&af->W, sizeof(double) * m * k));
    k_kernel_rows<T><<<nblk(m * k, 256), 256, 0, st>>>(wpd, P, n, af->F, m, af->L, k, pl->kernel,
                                                       pl->ell, sf2, Bf);
    k_times_lower_t<<<nblk(m * k, 256), 256, 0, st>>>(Bf, m, k, af->Ci, af->W);
    cudaFreeAsync(Bf, st);
    // pattern: FP64 window features of F, nearest earlier positions
    int pf = 0;
    for (int s = 0; s < P; ++s) pf += pl->win[s].d;
    double* xf = nullptr;
    AGP_CUDA(cudaMallocAsync(&xf, sizeof(double) * pf * m, st));
    for (int s = 0, c0 = 0; s < P; c0 += pl->win[s].d, ++s)
      k_gather_feat<T><<<nblk(m * pl->win[s].d, 256), 256, 0, st>>>(
          cp.xo[s], pl->win[s].d, n, af->F, m, c0, xf);
    AGP_CUDA(cudaMalloc(&af->J, sizeof(int32_t) * m * fill));
    AGP_CUDA(cudaMalloc(&af->len, sizeof(int32_t) * m));
    const size_t ksmem = kKnnWarps * knn_warp_bytes(pf);
    AGP_CUDA(cudaFuncSetAttribute(k_knn_lower, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ksmem));
    k_knn_lower<<<nblk(m, kKnnWarps), kKnnWarps * 32, ksmem, st>>>(xf, pf, m, fill, af->J,
                                                                   af->len);
    cudaFreeAsync(xf, st);
    // FSAI rows
    double* logdiag = nullptr;
    AGP_CUDA(cudaMallocAsync(&logdiag, sizeof(double) * m, st));
    AGP_CUDA(cudaMalloc(&af->Gval, sizeof(double) * m * fill));
    const size_t fsmem = sizeof(double) * (size_t)fill * (fill + 1);
    AGP_CUDA(cudaFuncSetAttribute(k_fsai_rows<T, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    k_fsai_rows<T, false><<<(unsigned)m, fsai_threads(fill), fsmem, st>>>(
        wpd, P, n, af->F, af->W, k, af->J, af->len, m, fill, pl->kernel, pl->ell, pl->sigma_f,
        pl->sigma_eps, af->Gval, logdiag, flag, nullptr, nullptr, nullptr, nullptr, nullptr);
    // G^T as compressed columns
    int32_t *cnt = nullptr, *cursor = nullptr;
    AGP_CUDA(cudaMallocAsync(&cnt, sizeof(int32_t) * m, st));
    AGP_CUDA(cudaMallocAsync(&cursor, sizeof(int32_t) * m, st));
    AGP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * m, st));
    AGP_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * m, st));
    AGP_CUDA(cudaMalloc(&af->colptr, sizeof(int32_t) * (m + 1)));
    k_col_count<<<nblk(m * fill, 256), 256, 0, st>>>(af->J, af->len, m, fill, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, af->colptr, m);
    int32_t nnz = 0;
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(&nnz, af->colptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    af->nnz = nnz;
    AGP_CUDA(cudaMalloc(&af->colrow, sizeof(int32_t) * std::max<int64_t>(1, nnz)));
    AGP_CUDA(cudaMalloc(&af->colval, sizeof(double) * std::max<int64_t>(1, nnz)));
    k_col_fill<<<nblk(m * fill, 256), 256, 0, st>>>(af->J, af->len, af->Gval, m, fill, af->colptr,
                                                    cursor, af->colrow, af->colval);
    std::vector<double> ld(m);
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(ld.data(), logdiag, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(logdiag, st);
    if (hflag) {
      cudaFreeAsync(flag, st);
      cudaFreeAsync(wpd, st);
      return set_error(AGP_ENAN, "AFN: a Schur complement block is not positive definite");
    }
    for (int64_t a = 0; a < m; ++a) logdet -= 2.0 * ld[a];
  }
  af->logdet = logdet;
  cudaFreeAsync(flag, st);
  cudaFreeAsync(wpd, st);
  // apply workspace
  af->slices = (int)std::min<int64_t>(256, std::max<int64_t>(1, (m + 2047) / 2048));
  af->rows_per_slice = std::max<int64_t>(1, (m + af->slices - 1) / af->slices);
  AGP_CUDA(cudaMalloc(&af->v, sizeof(double) * k * rmax));
  AGP_CUDA(cudaMalloc(&af->h, sizeof(double) * k * rmax));
  AGP_CUDA(cudaMalloc(&af->partial, sizeof(double) * af->slices * k * rmax));
  if (m > 0) {
    AGP_CUDA(cudaMalloc(&af->t, sizeof(double) * m * rmax));
    AGP_CUDA(cudaMalloc(&af->u, sizeof(double) * m * rmax));
    AGP_CUDA(cudaMalloc(&af->w, sizeof(double) * m * rmax));
  }
  AGP_CUDA(cudaMemsetAsync(af->partial, 0, sizeof(double) * af->slices * k * rmax, st));
  return cuda_status(cudaGetLastError(), "afn_build");
}

agp_status afn_apply(const Afn& af, const double* X, int64_t ldx, double* Y, int64_t ldy, int R,
                     cudaStream_t st) {
  if (R < 1 || R > af.rmax) return set_error(AGP_EINVAL, "AFN apply: too many columns");
  const int k = af.k;
  const int64_t m = af.m;
  k_afn_lm_in<<<nblk((int64_t)k * R, 128), 128, 0, st>>>(X, ldx, af.L, k, R, af.Ci, af.v);
  if (m > 0) {
    const unsigned blocks = (unsigned)std::min<int64_t>(nblk(m, 8), 152 * 16);
    const size_t smem = sizeof(double) * (size_t)k * R;
    AGP_CUDA(cudaFuncSetAttribute(k_afn_schur_in, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * kMaxLandmarkSet * 32)));
    k_afn_schur_in<<<blocks, 256, smem, st>>>(X, ldx, af.F, m, af.W, k, R, af.v, af.t);
    k_afn_g<<<blocks, 256, 0, st>>>(af.Gval, af.J, af.len, af.fill, m, R, af.t, af.u);
    k_afn_gt<<<blocks, 256, 0, st>>>(af.colptr, af.colrow, af.colval, m, R, af.u, af.w, af.F, Y,
                                     ldy);
    k_afn_wt<<<dim3((k + 31) / 32, af.slices), 256, 0, st>>>(af.W, af.w, m, k, R,
                                                            af.rows_per_slice, af.partial);
  }
  k_afn_lm_mid<<<nblk((int64_t)k * R, 128), 128, 0, st>>>(af.partial, m > 0 ? af.slices : 0, af.v,
                                                         k, R, af.h);
  k_afn_lm_out<<<nblk((int64_t)k * R, 128), 128, 0, st>>>(af.h, af.L, k, R, af.Ci, Y, ldy);
  return cuda_status(cudaGetLastError(), "afn_apply");
}

agp_status afn_pattern(const Afn& af, int32_t* landmarks, int32_t* J, cudaStream_t st) {
  if (landmarks) std::copy(af.landmarks.begin(), af.landmarks.end(), landmarks);
  if (J && af.m > 0) {
    AGP_CUDA(cudaMemcpyAsync(J, af.J, sizeof(int32_t) * af.m * af.fill, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
  }
  return AGP_OK;
}

// Derivative data for the likelihood gradient: host K_LL, C, C^{-1} and
// dK_LL/dell; Dl = (dK_FL/dell) C^{-T}; one pass of k_fsai_rows<T, true>
// (dG for ell, sigma_f, sigma_eps and the row sums G_t^T dS G_t); the levels
// of G for the forward substitution (row t depends on the earlier rows of
// its pattern: level(t) = 1 + the largest level among them).
template <typename T>
agp_status afn_build_derivs(agp_plan_s* pl, Afn* af, cudaStream_t st) {
  if (af->has_der) return AGP_OK;
  const int64_t n = pl->n, m = af->m;
  const int P = pl->P, k = af->k, fill = af->fill;
  const size_t kk = (size_t)k * k;
  const double sf2 = pl->sigma_f * pl->sigma_f, s2 = pl->sigma_eps * pl->sigma_eps;
  CallerPoints<T> cp;
  AGP_TRY(caller_points<T>(pl, cp, st));
  WinPts<T>* wpd = nullptr;
  double *Kd = nullptr, *Ed = nullptr, *Pd = nullptr, *logdiag = nullptr, *quad = nullptr;
  int* flag = nullptr;
  AGP_CUDA(cudaMallocAsync(&wpd, sizeof(WinPts<T>) * P, st));
  AGP_CUDA(cudaMemcpyAsync(wpd, cp.wp.data(), sizeof(WinPts<T>) * P, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMallocAsync(&Kd, sizeof(double) * kk, st));
  AGP_CUDA(cudaMallocAsync(&flag, sizeof(int), st));
  AGP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  struct Free {
    void** a;
    int na;
    cudaStream_t st;
    ~Free() {
      for (int i = 0; i < na; ++i)
        if (a[i]) cudaFreeAsync(a[i], st);
    }
  };
  void* tmp[7] = {wpd, Kd, flag, nullptr, nullptr, nullptr, nullptr};
  Free fr{tmp, 7, st};
  af->KLL_h.resize(kk);
  af->dKLL_h.resize(kk);
  af->C_h.resize(kk);
  af->Ci_h.resize(kk);
  k_kernel_block<T><<<nblk((int64_t)kk, 256), 256, 0, st>>>(wpd, P, n, af->L, k, pl->kernel,
                                                            pl->ell, sf2, 0, s2, Kd);
  AGP_CUDA(cudaMemcpyAsync(af->KLL_h.data(), Kd, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  k_kernel_block<T><<<nblk((int64_t)kk, 256), 256, 0, st>>>(wpd, P, n, af->L, k, pl->kernel,
                                                            pl->ell, sf2, 1, 0.0, Kd);
  AGP_CUDA(cudaMemcpyAsync(af->dKLL_h.data(), Kd, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaMemcpyAsync(af->C_h.data(), af->C, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaMemcpyAsync(af->Ci_h.data(), af->Ci, sizeof(double) * kk, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  af->quad_sum[0] = af->quad_sum[1] = af->quad_sum[2] = 0.0;
  if (m > 0) {
    // E = C^{-1} dK_LL C^{-T}, Pm = C^{-1} C^{-T} (host FP64)
    const std::vector<double>& Ci = af->Ci_h;
    std::vector<double> T1(kk), E(kk), Pm(kk);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double t = 0.0, p = 0.0;
        for (int q = 0; q <= i; ++q) t += Ci[(size_t)i * k + q] * af->dKLL_h[(size_t)q * k + j];
        for (int q = 0; q <= std::min(i, j); ++q) p += Ci[(size_t)i * k + q] * Ci[(size_t)j * k + q];
        T1[(size_t)i * k + j] = t;
        Pm[(size_t)i * k + j] = p;
      }
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        double t = 0.0;
        for (int q = 0; q <= j; ++q) t += T1[(size_t)i * k + q] * Ci[(size_t)j * k + q];
        E[(size_t)i * k + j] = t;
      }
    AGP_CUDA(cudaMallocAsync(&Ed, sizeof(double) * kk, st));
    AGP_CUDA(cudaMallocAsync(&Pd, sizeof(double) * kk, st));
    tmp[3] = Ed;
    tmp[4] = Pd;
    AGP_CUDA(cudaMemcpyAsync(Ed, E.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, st));
    AGP_CUDA(cudaMemcpyAsync(Pd, Pm.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, st));
    // Dl = (dK_FL/dell) C^{-T}
    double* Bf = nullptr;
    AGP_CUDA(cudaMallocAsync(&Bf, sizeof(double) * m * k, st));
    AGP_CUDA(cudaMalloc(&af->Dl, sizeof(double) * m * k));
    k_kernel_cols_rows<T><<<nblk(m * k, 256), 256, 0, st>>>(wpd, P, n, af->F, m, af->L, k,
                                                            pl->kernel, pl->ell, sf2, Bf);
    k_times_lower_t<<<nblk(m * k, 256), 256, 0, st>>>(Bf, m, k, af->Ci, af->Dl);
    cudaFreeAsync(Bf, st);
    // derivative rows of G
    AGP_CUDA(cudaMallocAsync(&logdiag, sizeof(double) * m, st));
    AGP_CUDA(cudaMallocAsync(&quad, sizeof(double) * 3 * m, st));
    tmp[5] = logdiag;
    tmp[6] = quad;
    AGP_CUDA(cudaMalloc(&af->dGval, sizeof(double) * 3 * m * fill));
    const size_t fsmem = sizeof(double) * (size_t)fill * (fill + 1);
    AGP_CUDA(cudaFuncSetAttribute(k_fsai_rows<T, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    k_fsai_rows<T, true><<<(unsigned)m, fsai_threads(fill), fsmem, st>>>(
        wpd, P, n, af->F, af->W, k, af->J, af->len, m, fill, pl->kernel, pl->ell, pl->sigma_f,
        pl->sigma_eps, af->Gval, logdiag, flag, af->Dl, Ed, Pd, af->dGval, quad);
    std::vector<double> qh(3 * m);
    int hflag = 0;
    AGP_CUDA(cudaGetLastError());
    AGP_CUDA(cudaMemcpyAsync(qh.data(), quad, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    // levels of the forward substitution
    std::vector<int32_t> Jh(m * fill), lenh(m);
    AGP_CUDA(cudaMemcpyAsync(Jh.data(), af->J, sizeof(int32_t) * m * fill, cudaMemcpyDeviceToHost,
                             st));
    AGP_CUDA(cudaMemcpyAsync(lenh.data(), af->len, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, st));
    AGP_CUDA(cudaStreamSynchronize(st));
    if (hflag) return set_error(AGP_ENAN, "AFN: a Schur complement block is not positive definite");
    for (int th = 0; th < 3; ++th)
      for (int64_t a = 0; a < m; ++a) af->quad_sum[th] += qh[(size_t)th * m + a];
    std::vector<int32_t> lev(m);
    int32_t depth = 0;
    for (int64_t t = 0; t < m; ++t) {
      int32_t l = 0;
      for (int q = 0; q < lenh[t] - 1; ++q) l = std::max(l, lev[Jh[(size_t)t * fill + q]] + 1);
      lev[t] = l;
      depth = std::max(depth, l + 1);
    }
    af->lvl_off.assign(depth + 1, 0);
    for (int64_t t = 0; t < m; ++t) ++af->lvl_off[lev[t] + 1];
    for (int32_t l = 0; l < depth; ++l) af->lvl_off[l + 1] += af->lvl_off[l];
    std::vector<int32_t> rows(m);
    std::vector<int64_t> cur(af->lvl_off.begin(), af->lvl_off.end() - 1);
    for (int64_t t = 0; t < m; ++t) rows[cur[lev[t]]++] = (int32_t)t;
    AGP_CUDA(cudaMalloc(&af->lvl_rows, sizeof(int32_t) * m));
    AGP_CUDA(cudaMemcpyAsync(af->lvl_rows, rows.data(), sizeof(int32_t) * m,
                             cudaMemcpyHostToDevice, st));
    AGP_CUDA(cudaStreamSynchronize(st));
  }
  af->has_der = true;
  return cuda_status(cudaGetLastError(), "afn_build_derivs");
}

agp_status afn_trsv(const Afn& af, const double* X, double* Y, int R, cudaStream_t st) {
  if (!af.has_der || R < 1 || R > 32) return set_error(AGP_EINVAL, "AFN: no levels / bad R");
  for (size_t l = 0; l + 1 < af.lvl_off.size(); ++l) {
    const int64_t nr = af.lvl_off[l + 1] - af.lvl_off[l];
    const unsigned blocks = (unsigned)std::min<int64_t>(nblk(nr, 8), 152 * 16);
    k_afn_trsv_level<<<blocks, 256, 0, st>>>(af.lvl_rows + af.lvl_off[l], nr, af.Gval, af.J, af.len,
                                             af.fill, R, X, Y);
  }
  return cuda_status(cudaGetLastError(), "afn_trsv");
}

agp_status afn_dg_apply(const Afn& af, int theta, const double* X, double* Y, int R,
                        cudaStream_t st) {
  if (!af.has_der || theta < 0 || theta > 2 || R < 1 || R > 32)
    return set_error(AGP_EINVAL, "AFN: no derivatives / bad arguments");
  if (af.m == 0) return AGP_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(nblk(af.m, 8), 152 * 16);
  k_afn_g<<<blocks, 256, 0, st>>>(af.dGval + (int64_t)theta * af.m * af.fill, af.J, af.len,
                                  af.fill, af.m, R, X, Y);
  return cuda_status(cudaGetLastError(), "afn_dg_apply");
}

agp_status afn_wt(const Afn& af, const double* A, const double* X, int R, double* out,
                  cudaStream_t st) {
  if (R < 1 || R > af.rmax) return set_error(AGP_EINVAL, "AFN: bad R");
  const int k = af.k;
  if (af.m == 0) {
    std::fill(out, out + (size_t)k * R, 0.0);
    return AGP_OK;
  }
  k_afn_wt<<<dim3((k + 31) / 32, af.slices), 256, 0, st>>>(A, X, af.m, k, R, af.rows_per_slice,
                                                          af.partial);
  k_sum_slices<<<nblk((int64_t)k * R, 128), 128, 0, st>>>(af.partial, af.slices, k, R, af.h);
  AGP_CUDA(cudaGetLastError());
  AGP_CUDA(cudaMemcpyAsync(out, af.h, sizeof(double) * k * R, cudaMemcpyDeviceToHost, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  return AGP_OK;
}

template agp_status afn_build_derivs<float>(agp_plan_s*, Afn*, cudaStream_t);
template agp_status afn_build_derivs<double>(agp_plan_s*, Afn*, cudaStream_t);
template agp_status afn_build<float>(agp_plan_s*, int, int, int, Afn*, cudaStream_t);
template agp_status afn_build<double>(agp_plan_s*, int, int, int, Afn*, cudaStream_t);

}  // namespace agp
