// pass_fs2_cols.cu - column steps of the four-step family.
#include "dct2d_launch.cuh"

namespace gbdct {
namespace {

template <int N1, int KIND>
cudaError_t col_launch(const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  using G = Fs2Geom<N1>;
  constexpr int S = (KIND == 0 || KIND == 3) ? G::B : G::A;
  using C = ColCfg<S>;
  const int nslab = (KIND == 0 || KIND == 3) ? G::A : G::B;
  if (prepare) {
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_colv<N1, KIND>),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  }
  k_fs2_colv<N1, KIND><<<dim3(nslab, a.n2 / 2 / C::COLS, batch), C::THREADS, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int N1>
cudaError_t cols_impl(int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (kind) {
    case 0: return col_launch<N1, 0>(a, batch, s, prepare);
    case 1: return col_launch<N1, 1>(a, batch, s, prepare);
    case 2: return col_launch<N1, 2>(a, batch, s, prepare);
    case 3: return col_launch<N1, 3>(a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fs2_col(int lg1, int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lg1) {
    case 8: return cols_impl<256>(kind, a, batch, s, prepare);
    case 9: return cols_impl<512>(kind, a, batch, s, prepare);
    case 10: return cols_impl<1024>(kind, a, batch, s, prepare);
    case 11: return cols_impl<2048>(kind, a, batch, s, prepare);
    case 12: return cols_impl<4096>(kind, a, batch, s, prepare);
    case 13: return cols_impl<8192>(kind, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbdct
