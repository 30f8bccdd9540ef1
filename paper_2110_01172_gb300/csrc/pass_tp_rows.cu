// pass_tp_rows.cu - row passes of the two-pass family (radix-2 column step
// folded into the loads / stores), and the whole-transform launcher
// (forward: column pass, row pass; inverse: row pass, column pass).
#include "dct2d_launch.cuh"
#include "dct2d_tp_kernels.cuh"

namespace gbdct {
namespace {

template <int L, bool NARROW>
cudaError_t row_launch_g(bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  using R = TpRows<L, NARROW>;
  if (prepare) {
    const void* plain[] = {reinterpret_cast<const void*>(k_tp_rows_fwd<L, NARROW>),
                           reinterpret_cast<const void*>(k_tp_rows_inv<L, false, false, NARROW>),
                           reinterpret_cast<const void*>(k_tp_rows_inv<L, true, false, NARROW>)};
    const void* staged[] = {reinterpret_cast<const void*>(k_tp_rows_inv<L, false, true, NARROW>),
                            reinterpret_cast<const void*>(k_tp_rows_inv<L, true, true, NARROW>)};
    cudaError_t e = cudaSuccess;
    for (const void* k : plain)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM);
    for (const void* k : staged)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R::SMEM_STAGED);
    return e;
  }
  if ((a.n1 / 4) % R::NP) return cudaErrorInvalidValue;
  const dim3 grid(a.n1 / 4 / R::NP, 1, batch);
  // device input: the inverse's rows are staged by bulk copies; host-mapped input: read directly
  const bool mapped = a.vkind == 1 || a.vkind == 2;
  if (inverse && a.io_dev && mapped)
    return pdl::launch(k_tp_rows_inv<L, true, true, NARROW>, grid, dim3(R::THREADS), R::SMEM_STAGED, s, a);
  else if (inverse && a.io_dev)
    return pdl::launch(k_tp_rows_inv<L, false, true, NARROW>, grid, dim3(R::THREADS), R::SMEM_STAGED, s, a);
  else if (inverse && mapped)
    return pdl::launch(k_tp_rows_inv<L, true, false, NARROW>, grid, dim3(R::THREADS), R::SMEM, s, a);
  else if (inverse)
    return pdl::launch(k_tp_rows_inv<L, false, false, NARROW>, grid, dim3(R::THREADS), R::SMEM, s, a);
  else
    return pdl::launch(k_tp_rows_fwd<L, NARROW>, grid, dim3(R::THREADS), R::SMEM, s, a);
}

// Narrow (64-thread) CTAs when wide ones would give fewer than two CTAs per SM.
template <int L>
cudaError_t row_launch(bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if (prepare) {
    cudaError_t e = row_launch_g<L, false>(inverse, a, batch, s, true);
    if (e == cudaSuccess) e = row_launch_g<L, true>(inverse, a, batch, s, true);
    return e;
  }
  const long long wide_ctas = (long long)(a.n1 / 4 / TpRows<L, false>::NP) * batch;
  if (wide_ctas < 2LL * (a.nsm > 0 ? a.nsm : 1) && (a.n1 / 4) % TpRows<L, true>::NP == 0)
    return row_launch_g<L, true>(inverse, a, batch, s, false);
  return row_launch_g<L, false>(inverse, a, batch, s, false);
}

cudaError_t run_rows(int lg2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lg2) {
    case 7: return row_launch<128>(inverse, a, batch, s, prepare);
    case 8: return row_launch<256>(inverse, a, batch, s, prepare);
    case 9: return row_launch<512>(inverse, a, batch, s, prepare);
    case 10: return row_launch<1024>(inverse, a, batch, s, prepare);
    case 11: return row_launch<2048>(inverse, a, batch, s, prepare);
    case 12: return row_launch<4096>(inverse, a, batch, s, prepare);
    case 13: return row_launch<8192>(inverse, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t run_tp(int lg1, int lg2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if (prepare) {
    cudaError_t e = run_rows(lg2, false, a, batch, s, true);
    if (e == cudaSuccess) e = run_tp_cols(lg1, false, a, batch, s, true);
    return e;
  }
  const int f = a.step_filter;
  cudaError_t e = cudaSuccess;
  if (!inverse) {
    if (f < 0 || f == 0) e = run_tp_cols(lg1, false, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = run_rows(lg2, false, a, batch, s, false);
  } else {
    if (f < 0 || f == 0) e = run_rows(lg2, true, a, batch, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = run_tp_cols(lg1, true, a, batch, s, false);
  }
  return e;
}

}  // namespace gbdct
