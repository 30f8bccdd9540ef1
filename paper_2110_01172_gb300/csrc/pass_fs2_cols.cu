// pass_fs2_cols.cu - column steps of the four-step family.
#include "dct2d_launch.cuh"

namespace gbdct {
namespace {

template <int N1, int A, int KIND>
cudaError_t col_launch(const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  using G = Fs2Geom<N1, A>;
  constexpr int S = (KIND == 0 || KIND == 3) ? G::B : G::A;
  using C = ColCfg<S>;
  const int nslab = (KIND == 0 || KIND == 3) ? G::A : G::B;
  if (prepare) {
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_colv<N1, A, KIND>),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  }
  k_fs2_colv<N1, A, KIND><<<dim3(nslab, a.n2 / 2 / C::COLS, batch), C::THREADS, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int N1, int A>
cudaError_t cols_impl(int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if constexpr (A >= 16 && A <= 128 && N1 / A >= 16 && N1 / A <= 128) {
    switch (kind) {
      case 0: return col_launch<N1, A, 0>(a, batch, s, prepare);
      case 1: return col_launch<N1, A, 1>(a, batch, s, prepare);
      case 2: return col_launch<N1, A, 2>(a, batch, s, prepare);
      case 3: return col_launch<N1, A, 3>(a, batch, s, prepare);
    }
  }
  return cudaErrorInvalidValue;
}

template <int N1>
cudaError_t cols_split(int A, int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (A) {
    case 16: return cols_impl<N1, 16>(kind, a, batch, s, prepare);
    case 32: return cols_impl<N1, 32>(kind, a, batch, s, prepare);
    case 64: return cols_impl<N1, 64>(kind, a, batch, s, prepare);
    case 128: return cols_impl<N1, 128>(kind, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fs2_col(int lg1, int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lg1) {
    case 8: return cols_split<256>(a.fsA, kind, a, batch, s, prepare);
    case 9: return cols_split<512>(a.fsA, kind, a, batch, s, prepare);
    case 10: return cols_split<1024>(a.fsA, kind, a, batch, s, prepare);
    case 11: return cols_split<2048>(a.fsA, kind, a, batch, s, prepare);
    case 12: return cols_split<4096>(a.fsA, kind, a, batch, s, prepare);
    case 13: return cols_split<8192>(a.fsA, kind, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbdct
