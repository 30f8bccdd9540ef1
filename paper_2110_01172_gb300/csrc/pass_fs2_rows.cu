// pass_fs2_rows.cu - row passes of the occupancy-first four-step family, and
// the whole-transform launcher (forward: C1, C2, rows; inverse: rows, C2', C1').
#include "dct2d_launch.cuh"

namespace gbdct {

namespace {

template <int L>
cudaError_t row_launch(bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if constexpr (L <= 8192) {  // two items per thread group (packed two-lane arithmetic)
    using R = RowX2Geom<L>;
    if (prepare) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_rows_fwd_x2<L>),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_rows_inv_x2<L, false>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_rows_inv_x2<L, true>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
      return e;
    }
    const dim3 grid(a.n1 / 4 / R::NP, 1, batch);
    if (inverse && (a.vkind == 1 || a.vkind == 2))
      k_fs2_rows_inv_x2<L, true><<<grid, R::THREADS, R::SMEM, s>>>(a);
    else if (inverse)
      k_fs2_rows_inv_x2<L, false><<<grid, R::THREADS, R::SMEM, s>>>(a);
    else
      k_fs2_rows_fwd_x2<L><<<grid, R::THREADS, R::SMEM, s>>>(a);
    return cudaGetLastError();
  } else {
    using R = RowGeom<L>;
    if (prepare) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_rows<L, false>),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_fs2_rows<L, true>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
      return e;
    }
    const dim3 grid(a.n1 / 2 / R::NI, 1, batch);
    if (inverse)
      k_fs2_rows<L, true><<<grid, R::THREADS, R::SMEM, s>>>(a);
    else
      k_fs2_rows<L, false><<<grid, R::THREADS, R::SMEM, s>>>(a);
    return cudaGetLastError();
  }
}

cudaError_t run_rows(int lg2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lg2) {
    case 8: return row_launch<256>(inverse, a, batch, s, prepare);
    case 9: return row_launch<512>(inverse, a, batch, s, prepare);
    case 10: return row_launch<1024>(inverse, a, batch, s, prepare);
    case 11: return row_launch<2048>(inverse, a, batch, s, prepare);
    case 12: return row_launch<4096>(inverse, a, batch, s, prepare);
    case 13: return row_launch<8192>(inverse, a, batch, s, prepare);
    case 14: return row_launch<16384>(inverse, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_fs2(int lg1, int lg2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if (prepare) {
    cudaError_t e = run_rows(lg2, false, a, batch, s, true);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = run_fs2_col(lg1, k, a, batch, s, true);
    return e;
  }
  const int f = a.step_filter;
  cudaError_t e = cudaSuccess;
  if (!inverse) {
    if (f < 0 || f == 0) e = run_fs2_col(lg1, 0, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = run_fs2_col(lg1, 1, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 2)) e = run_rows(lg2, false, a, batch, s, false);
  } else {
    if (f < 0 || f == 0) e = run_rows(lg2, true, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = run_fs2_col(lg1, 2, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 2)) e = run_fs2_col(lg1, 3, a, batch, s, false);
  }
  return e;
}

}  // namespace gbdct
