// Batches of independent problems: one launch per matvec stage for all
// problems of a batch (independent GP problems of uneven size, each with its
// own plan and hyperparameters).
//
// The batch concatenates the plans' window tables (WinDev), their work items
// (window index remapped into the combined table, grouped by window
// dimension) and their DFT buffer tables (grouped by (d, N)); per-window
// right-hand sides, outputs and scale factors come from a WinIO table filled
// by agp_batch_bind. agp_batch_matvec then enqueues: output init (one launch
// over all problems), grid zeroing, spreading, the DFT stages and
// interpolation -- a fixed kernel sequence with no host synchronisation.
#include <new>
#include <vector>

#include "agp_internal.cuh"

namespace agp {
namespace {

template <typename T>
struct ProbIO {
  const T* V;
  int64_t ldv;
  T* Out;
  int64_t ldo;
  int64_t n;
  T noise_mv;    // sigma_eps^2 (K_hat)
  T noise_se;    // 2 sigma_eps (dK/dsigma_eps)
};

// Out_q = noise_q V_q for every problem q (blockIdx.y = q)
template <typename T>
__global__ void k_batch_init(const ProbIO<T>* __restrict__ probs, int R, int which) {
  const ProbIO<T> p = probs[blockIdx.y];
  const T a = (which == -1) ? p.noise_mv : ((which == AGP_D_SIGMA_EPS) ? p.noise_se : T(0));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < p.n * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    p.Out[i * p.ldo + r] = (a == T(0)) ? T(0) : a * p.V[i * p.ldv + r];
  }
}

__global__ void k_remap_items(const int4* __restrict__ src, int64_t n, int offset,
                              int4* __restrict__ dst) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  int4 v = src[e];
  v.x += offset;
  dst[e] = v;
}

}  // namespace
}  // namespace agp

struct agp_batch_s {
  int nprob = 0;
  agp_prec prec = AGP_F32;
  int s = 0;
  int R = 0, rc = 0;
  bool bound = false;
  std::vector<agp_plan> plans;
  std::vector<int> win_offset;       // first combined window of each problem
  int nwin = 0;
  void* wins_dev = nullptr;          // WinDev<T>[nwin]
  int4* items = nullptr;             // combined items, grouped by d
  int64_t items_by_d[agp::kMaxDim + 1] = {0, 0, 0, 0};
  std::vector<agp::FftGroup> groups; // combined DFT groups
  void* io_k = nullptr;              // WinIO<T>[nwin], scale sigma_f^2
  void* io_sf = nullptr;             // WinIO<T>[nwin], scale 2 sigma_f
  void* probs = nullptr;             // ProbIO<T>[nprob]
  int64_t nmax = 0;
};

namespace agp {
namespace {

#define AGP_CUDA(call)                                             \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_status(e_, #call);          \
  } while (0)

void free_batch(agp_batch_s* b) {
  if (!b) return;
  cudaFree(b->wins_dev);
  cudaFree(b->items);
  for (auto& g : b->groups) cudaFree(g.tab);
  cudaFree(b->io_k);
  cudaFree(b->io_sf);
  cudaFree(b->probs);
  delete b;
}

template <typename T>
agp_status batch_build(agp_batch_s* b, cudaStream_t st) {
  // combined window table
  std::vector<WinDev<T>> wd;
  std::vector<FftWin> fw;
  for (int q = 0; q < b->nprob; ++q) {
    const agp_plan_s* pl = b->plans[q];
    b->win_offset.push_back((int)wd.size());
    for (const Window& w : pl->win) {
      WinDev<T> d;
      d.xs = reinterpret_cast<const T*>(w.xs);
      d.perm = w.perm;
      d.wts = reinterpret_cast<const T*>(w.wts);
      d.grid = reinterpret_cast<T*>(w.grid);
      d.cell_start = w.cell_start;
      d.n = pl->n;
      d.N = w.N;
      d.n_os = w.n_os;
      d.W = w.W;
      wd.push_back(d);
      fw.push_back(FftWin{w.grid, w.specA, w.specB, w.tw, w.dmul, w.dmul_der});
    }
    b->nmax = std::max<int64_t>(b->nmax, pl->n);
  }
  b->nwin = (int)wd.size();
  AGP_CUDA(cudaMalloc(&b->wins_dev, sizeof(WinDev<T>) * b->nwin));
  AGP_CUDA(cudaMemcpyAsync(b->wins_dev, wd.data(), sizeof(WinDev<T>) * b->nwin,
                           cudaMemcpyHostToDevice, st));
  // combined items grouped by d
  int64_t total = 0;
  for (auto* pl : b->plans) total += pl->items_by_d[kMaxDim];
  AGP_CUDA(cudaMalloc(&b->items, sizeof(int4) * std::max<int64_t>(1, total)));
  int64_t off = 0;
  for (int dd = 1; dd <= kMaxDim; ++dd) {
    b->items_by_d[dd - 1] = off;
    for (int q = 0; q < b->nprob; ++q) {
      const agp_plan_s* pl = b->plans[q];
      const int64_t a = pl->items_by_d[dd - 1], e = pl->items_by_d[dd];
      if (e == a) continue;
      k_remap_items<<<(unsigned)((e - a + 255) / 256), 256, 0, st>>>(pl->items_all + a, e - a,
                                                                     b->win_offset[q], b->items + off);
      off += e - a;
    }
  }
  b->items_by_d[kMaxDim] = off;
  AGP_CUDA(cudaGetLastError());
  // combined DFT groups by (d, N)
  std::vector<std::vector<FftWin>> gtab;
  int k = 0;
  for (int q = 0; q < b->nprob; ++q) {
    for (const Window& w : b->plans[q]->win) {
      size_t gi = 0;
      while (gi < b->groups.size() && !(b->groups[gi].d == w.d && b->groups[gi].N == w.N)) ++gi;
      if (gi == b->groups.size()) {
        FftGroup g = w.self_group();
        g.count = 0;
        g.tab = nullptr;
        b->groups.push_back(g);
        gtab.emplace_back();
      }
      b->groups[gi].count += 1;
      gtab[gi].push_back(fw[k++]);
    }
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    AGP_CUDA(cudaMalloc(&b->groups[gi].tab, sizeof(FftWin) * gtab[gi].size()));
    AGP_CUDA(cudaMemcpyAsync(b->groups[gi].tab, gtab[gi].data(), sizeof(FftWin) * gtab[gi].size(),
                             cudaMemcpyHostToDevice, st));
  }
  AGP_CUDA(cudaMalloc(&b->io_k, sizeof(WinIO<T>) * b->nwin));
  AGP_CUDA(cudaMalloc(&b->io_sf, sizeof(WinIO<T>) * b->nwin));
  AGP_CUDA(cudaMalloc(&b->probs, sizeof(ProbIO<T>) * b->nprob));
  AGP_CUDA(cudaStreamSynchronize(st));   // host tables go out of scope
  return AGP_OK;
}

template <typename T>
agp_status batch_bind(agp_batch_s* b, const void* const* V, const int64_t* ldv, void* const* Out,
                      const int64_t* ldo, int R, cudaStream_t st) {
  std::vector<WinIO<T>> iok(b->nwin), iosf(b->nwin);
  std::vector<ProbIO<T>> pr(b->nprob);
  for (int q = 0; q < b->nprob; ++q) {
    const agp_plan_s* pl = b->plans[q];
    const T* v = reinterpret_cast<const T*>(V[q]);
    T* o = reinterpret_cast<T*>(Out[q]);
    pr[q] = ProbIO<T>{v, ldv[q], o, ldo[q], pl->n, (T)(pl->sigma_eps * pl->sigma_eps),
                      (T)(2.0 * pl->sigma_eps)};
    for (int s = 0; s < pl->P; ++s) {
      iok[b->win_offset[q] + s] = WinIO<T>{v, ldv[q], o, ldo[q], (T)(pl->sigma_f * pl->sigma_f)};
      iosf[b->win_offset[q] + s] = WinIO<T>{v, ldv[q], o, ldo[q], (T)(2.0 * pl->sigma_f)};
    }
  }
  AGP_CUDA(cudaMemcpyAsync(b->io_k, iok.data(), sizeof(WinIO<T>) * b->nwin, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMemcpyAsync(b->io_sf, iosf.data(), sizeof(WinIO<T>) * b->nwin, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaMemcpyAsync(b->probs, pr.data(), sizeof(ProbIO<T>) * b->nprob, cudaMemcpyHostToDevice, st));
  AGP_CUDA(cudaStreamSynchronize(st));
  return AGP_OK;
}

template <typename T>
agp_status batch_matvec(agp_batch_s* b, int which, cudaStream_t st) {
  const unsigned bx = (unsigned)std::min<int64_t>((b->nmax * b->R + 255) / 256, 4096);
  k_batch_init<T><<<dim3(bx, b->nprob), 256, 0, st>>>(reinterpret_cast<const ProbIO<T>*>(b->probs),
                                                     b->R, which);
  AGP_CUDA(cudaGetLastError());
  if (which == AGP_D_SIGMA_EPS) return AGP_OK;
  const WinDev<T>* wins = reinterpret_cast<const WinDev<T>*>(b->wins_dev);
  const WinIO<T>* io = reinterpret_cast<const WinIO<T>*>(which == AGP_D_SIGMA_F ? b->io_sf : b->io_k);
  const int der = which == AGP_D_ELL;
  for (const auto& g : b->groups) AGP_CUDA(zero_grids<T>(g, b->rc, st));
  for (int dd = 1; dd <= kMaxDim; ++dd) {
    const int64_t a = b->items_by_d[dd - 1], e = b->items_by_d[dd];
    if (e > a)
      AGP_CUDA(spread_items_sel<T>(wins, io, b->items + a, e - a, dd, b->s, b->rc, nullptr, 0,
                                   b->R, b->plans[0]->use_tc, b->plans[0]->err_dev,
                                   b->plans[0]->wait_limit, st));
  }
  // groups with d = 2 or 3: the three-launch DFT stage; the others per group
  FftGroup fg[8];
  int nf = 0;
  for (const auto& g : b->groups)
    if (dft_fused_supported(g) && nf < 8) fg[nf++] = g;
  if (nf > 0) AGP_CUDA(dft_stage<T>(fg, nf, der, b->rc, st));
  for (const auto& g : b->groups) {
    bool done = false;
    for (int q = 0; q < nf; ++q) done = done || fg[q].tab == g.tab;
    if (done) continue;
    AGP_CUDA(fft_forward<T>(g, b->rc, st));
    AGP_CUDA(spectral_multiply<T>(g, der, b->rc, st));
    AGP_CUDA(fft_inverse<T>(g, b->rc, st));
  }
  for (int dd = 1; dd <= kMaxDim; ++dd) {
    const int64_t a = b->items_by_d[dd - 1], e = b->items_by_d[dd];
    if (e > a)
      AGP_CUDA(interp_items_sel<T>(wins, io, b->items + a, e - a, dd, b->s, b->rc, nullptr, 0,
                                   b->R, T(0), b->plans[0]->use_tc, b->plans[0]->err_dev,
                                   b->plans[0]->wait_limit, st));
  }
  return AGP_OK;
}

}  // namespace
}  // namespace agp

using namespace agp;

extern "C" {

agp_status agp_batch_create(agp_batch* out, const agp_plan* plans, int nprob, void* stream) {
  if (!out) return set_error(AGP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!plans || nprob < 1) return set_error(AGP_EINVAL, "need nprob >= 1 plans");
  for (int q = 0; q < nprob; ++q) {
    if (!plans[q]) return set_error(AGP_EINVAL, "NULL plan in batch");
    if (plans[q]->prec != plans[0]->prec || plans[q]->s != plans[0]->s)
      return set_error(AGP_EINVAL, "batched plans must share precision and cutoff");
    if (plans[q]->use_tc != plans[0]->use_tc)
      return set_error(AGP_EINVAL, "batched plans must share the tensor-core setting");
  }
  auto* b = new (std::nothrow) agp_batch_s();
  if (!b) return set_error(AGP_ENOMEM, "host allocation");
  b->nprob = nprob;
  b->prec = plans[0]->prec;
  b->s = plans[0]->s;
  b->plans.assign(plans, plans + nprob);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  agp_status s = b->prec == AGP_F32 ? batch_build<float>(b, st) : batch_build<double>(b, st);
  if (s != AGP_OK) {
    cudaStreamSynchronize(st);
    free_batch(b);
    return s;
  }
  *out = b;
  return AGP_OK;
}

agp_status agp_batch_destroy(agp_batch b) {
  if (!b) return AGP_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_batch(b);
  return cuda_status(e, "agp_batch_destroy");
}

agp_status agp_batch_bind(agp_batch b, const void* const* V, const int64_t* ldv, void* const* Out,
                          const int64_t* ldo, int R, void* stream) {
  if (!b || !V || !ldv || !Out || !ldo) return set_error(AGP_EINVAL, "bad arguments");
  const int rmax = b->prec == AGP_F32 ? 32 : 4;
  if (R < 1 || R > rmax) return set_error(AGP_EINVAL, "R out of range for a batch");
  for (int q = 0; q < b->nprob; ++q) {
    if (!V[q] || !Out[q] || ldv[q] < R || ldo[q] < R)
      return set_error(AGP_EINVAL, "bad V/Out of a batched problem");
    const size_t es = b->prec == AGP_F32 ? 4 : 8;
    const char* v0 = static_cast<const char*>(V[q]);
    const char* o0 = static_cast<const char*>(Out[q]);
    const int64_t n = b->plans[q]->n;
    if (v0 < o0 + es * (size_t)((n - 1) * ldo[q] + R) && o0 < v0 + es * (size_t)((n - 1) * ldv[q] + R))
      return set_error(AGP_EINVAL, "Out overlaps V in a batched problem");
  }
  b->R = R;
  b->rc = rhs_block_width(b->prec, R);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  agp_status s = b->prec == AGP_F32 ? batch_bind<float>(b, V, ldv, Out, ldo, R, st)
                                    : batch_bind<double>(b, V, ldv, Out, ldo, R, st);
  b->bound = s == AGP_OK;
  return s;
}

agp_status agp_batch_matvec(agp_batch b, int which, void* stream) {
  if (!b || !b->bound) return set_error(AGP_EINVAL, "batch not bound");
  if (which < -1 || which > AGP_D_SIGMA_EPS) return set_error(AGP_EINVAL, "bad which");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return b->prec == AGP_F32 ? batch_matvec<float>(b, which, st) : batch_matvec<double>(b, which, st);
}

}  // extern "C"
