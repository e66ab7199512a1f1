// Dispatch of spreading and interpolation over the right-hand-side block
// width; the kernels are in agp_nufft_kernels.cuh, instantiated per width in
// agp_nufft_rc<RC>.cu.
#include "agp_nufft_kernels.cuh"

namespace agp {

template <typename T>
cudaError_t spread_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, const T* V, int64_t ldv, int R,
                         cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    switch (RC) {
      case 32: return spread_rc32(wins, io, items, n_items, d, s, V, ldv, R, st);
      case 24: return spread_rc24(wins, io, items, n_items, d, s, V, ldv, R, st);
      case 16: return spread_rc16(wins, io, items, n_items, d, s, V, ldv, R, st);
      case 8: return spread_rc8(wins, io, items, n_items, d, s, V, ldv, R, st);
      case 1: return spread_rc1(wins, io, items, n_items, d, s, V, ldv, R, st);
    }
  } else {
    switch (RC) {
      case 4: return spread_rc4(wins, io, items, n_items, d, s, V, ldv, R, st);
      case 1: return spread_rc1(wins, io, items, n_items, d, s, V, ldv, R, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t interp_items(const WinDev<T>* wins, const WinIO<T>* io, const int4* items,
                         int64_t n_items, int d, int s, int RC, T* Out, int64_t ldo, int R,
                         T scale, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    switch (RC) {
      case 32: return interp_rc32(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
      case 24: return interp_rc24(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
      case 16: return interp_rc16(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
      case 8: return interp_rc8(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
      case 1: return interp_rc1(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
    }
  } else {
    switch (RC) {
      case 4: return interp_rc4(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
      case 1: return interp_rc1(wins, io, items, n_items, d, s, Out, ldo, R, scale, st);
    }
  }
  return cudaErrorInvalidValue;
}

int rhs_block_width(agp_prec prec, int R) {
  if (prec == AGP_F32) return R >= 25 ? 32 : R >= 17 ? 24 : R >= 9 ? 16 : R >= 2 ? 8 : 1;
  return R >= 2 ? 4 : 1;
}

template cudaError_t spread_items<float>(const WinDev<float>*, const WinIO<float>*, const int4*,
                                         int64_t, int, int, int, const float*, int64_t, int,
                                         cudaStream_t);
template cudaError_t spread_items<double>(const WinDev<double>*, const WinIO<double>*, const int4*,
                                          int64_t, int, int, int, const double*, int64_t, int,
                                          cudaStream_t);
template cudaError_t interp_items<float>(const WinDev<float>*, const WinIO<float>*, const int4*,
                                         int64_t, int, int, int, float*, int64_t, int, float,
                                         cudaStream_t);
template cudaError_t interp_items<double>(const WinDev<double>*, const WinIO<double>*, const int4*,
                                          int64_t, int, int, int, double*, int64_t, int, double,
                                          cudaStream_t);

}  // namespace agp
