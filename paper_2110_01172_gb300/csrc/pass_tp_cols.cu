// pass_tp_cols.cu - column passes of the two-pass family (half-length column
// FFTs of the even and odd reordered rows).
#include "dct2d_launch.cuh"
#include "dct2d_tp_kernels.cuh"

namespace gbdct {
namespace {

// Tensor maps of the bulk-copy column pass: mx over the input (forward) or
// output (inverse) viewed as (x, row % 4, row / 4, batch), mw over the
// workspace (x, row, batch); boxes of 4 NP floats x ZB rows.
bool encode_maps(const Dct2dArgs& a, int batch, bool inverse, int np, int zb, CUtensorMap* mx, CUtensorMap* mw) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tma::encoder();
  if (!fn) return false;
  const cuuint64_t n1 = (cuuint64_t)a.n1, n2 = (cuuint64_t)a.n2;
  void* xp = inverse ? static_cast<void*>(a.out) : const_cast<float*>(a.in);
  const cuuint64_t dx[4] = {n2, 4, n1 / 4, (cuuint64_t)batch};
  const cuuint64_t sx[3] = {n2 * 4, 16 * n2, (cuuint64_t)(inverse ? a.out_bstride : a.in_bstride) * 4};
  const cuuint32_t bx[4] = {(cuuint32_t)(4 * np), 1, (cuuint32_t)zb, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  if (fn(mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, xp, dx, sx, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t dw[3] = {n2, n1, (cuuint64_t)batch};
  const cuuint64_t sw[2] = {n2 * 4, (cuuint64_t)a.work_bstride * 8};
  const cuuint32_t bw[3] = {(cuuint32_t)(4 * np), (cuuint32_t)zb, 1};
  return fn(mw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.work, dw, sw, bw, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <int M, int NP>
cudaError_t col_launch(bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  using G = TpColGeom<M, NP>;
  if constexpr (!G::VALID) {
    return cudaErrorInvalidValue;
  } else {
    if (prepare) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_tp_cols<M, NP, false>),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_tp_cols<M, NP, true>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_tp_cols_tma<M, NP, false>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_TMA);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_tp_cols_tma<M, NP, true>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_TMA);
      return e;
    }
    if ((a.n2 / 4) % NP) return cudaErrorInvalidValue;
    const dim3 grid(a.n2 / 4 / NP, 2, batch);
    // bulk tensor copies for device buffers; per-thread loads / stores for
    // host-mapped or managed buffers
    CUtensorMap mx, mw;
    if (a.io_dev && encode_maps(a, batch, inverse, NP, G::ZB, &mx, &mw)) {
      if (inverse)
        return pdl::launch(k_tp_cols_tma<M, NP, true>, grid, dim3(G::THREADS), G::SMEM_TMA, s, a, mx, mw);
      else
        return pdl::launch(k_tp_cols_tma<M, NP, false>, grid, dim3(G::THREADS), G::SMEM_TMA, s, a, mx, mw);
    }
    if (inverse)
      return pdl::launch(k_tp_cols<M, NP, true>, grid, dim3(G::THREADS), G::SMEM, s, a);
    else
      return pdl::launch(k_tp_cols<M, NP, false>, grid, dim3(G::THREADS), G::SMEM, s, a);
  }
}

// The strip width: the plan's choice, else the default for M, halved (down
// to two column pairs and 64 threads) while the grid would give fewer than
// two CTAs per SM (a single transform with few columns, e.g. 1024^2).
template <int M>
int strip_np(const Dct2dArgs& a, int batch) {
  if (a.tpNP) return a.tpNP;
  int np = tp_default_np(M);
  const long long nsm = a.nsm > 0 ? a.nsm : 1;
  while (np > 2 && (np / 2) * fft_tps(M) >= 64 && (long long)(a.n2 / 4 / np) * 2 * batch < 2 * nsm) np /= 2;
  return np;
}

template <int M>
cudaError_t col_np(bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  if (prepare) {  // every width the default or the grid rule can pick
    cudaError_t e = cudaSuccess;
    for (int np = (a.tpNP ? a.tpNP : tp_default_np(M)); np >= 1 && e == cudaSuccess; np /= 2) {
      switch (np) {
        case 1: e = col_launch<M, 1>(inverse, a, batch, s, true); break;
        case 2: e = col_launch<M, 2>(inverse, a, batch, s, true); break;
        case 4: e = col_launch<M, 4>(inverse, a, batch, s, true); break;
        case 8: e = col_launch<M, 8>(inverse, a, batch, s, true); break;
        case 16: e = col_launch<M, 16>(inverse, a, batch, s, true); break;
        case 32: e = col_launch<M, 32>(inverse, a, batch, s, true); break;
      }
      if (e == cudaErrorInvalidValue) e = cudaSuccess;  // width not built for this M
      if (a.tpNP) break;
    }
    return e;
  }
  switch (strip_np<M>(a, batch)) {  // strip width in column pairs
    case 1: return col_launch<M, 1>(inverse, a, batch, s, prepare);
    case 2: return col_launch<M, 2>(inverse, a, batch, s, prepare);
    case 4: return col_launch<M, 4>(inverse, a, batch, s, prepare);
    case 8: return col_launch<M, 8>(inverse, a, batch, s, prepare);
    case 16: return col_launch<M, 16>(inverse, a, batch, s, prepare);
    case 32: return col_launch<M, 32>(inverse, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

// a.tpNP: the strip width NP in column pairs (0: the default for M).
cudaError_t run_tp_cols(int lg1, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lg1) {  // M = N1 / 2
    case 7: return col_np<64>(inverse, a, batch, s, prepare);
    case 8: return col_np<128>(inverse, a, batch, s, prepare);
    case 9: return col_np<256>(inverse, a, batch, s, prepare);
    case 10: return col_np<512>(inverse, a, batch, s, prepare);
    case 11: return col_np<1024>(inverse, a, batch, s, prepare);
    case 12: return col_np<2048>(inverse, a, batch, s, prepare);
    case 13: return col_np<4096>(inverse, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbdct
