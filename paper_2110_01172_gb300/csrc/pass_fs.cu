// pass_fs.cu - launches of the four-step family (column steps + row passes).
#include "dct2d_launch.cuh"

namespace gbdct {
namespace {

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <int N1, int N2>
cudaError_t fs_impl(bool inverse, const Dct2dArgs& a, const float2* fstw, int batch, cudaStream_t s,
                    bool prepare) {
  using G = FsGeom<N1>;
  using R = R64Geom<N2>;
  const dim3 g1(G::A, N2 / 2 / kFsCols, batch), g2(G::B, N2 / 2 / kFsCols, batch);
  const dim3 gr(N1 / 4, 1, batch);
  if (prepare) {
    cudaError_t e = set_smem(k_fs_fwd_c1<N1>, G::SMEM);
    if (e == cudaSuccess) e = set_smem(k_fs_c2<N1, false>, G::SMEM);
    if (e == cudaSuccess) e = set_smem(k_fs_c2<N1, true>, G::SMEM);
    if (e == cudaSuccess) e = set_smem(k_fs_inv_c1<N1>, G::SMEM);
    if (e == cudaSuccess) e = set_smem(k_fs_fwd_rows<N1, N2>, R::SMEM);
    if (e == cudaSuccess) e = set_smem(k_fs_inv_rows<N1, N2>, R::SMEM);
    return e;
  }
  const int f = a.step_filter;
  if (!inverse) {
    if (f < 0 || f == 0) k_fs_fwd_c1<N1><<<g1, kFsCols, G::SMEM, s>>>(a, fstw);
    if (f < 0 || f == 1) k_fs_c2<N1, false><<<g2, kFsCols, G::SMEM, s>>>(a, fstw);
    if (f < 0 || f == 2) k_fs_fwd_rows<N1, N2><<<gr, R::THREADS, R::SMEM, s>>>(a);
  } else {
    if (f < 0 || f == 0) k_fs_inv_rows<N1, N2><<<gr, R::THREADS, R::SMEM, s>>>(a);
    if (f < 0 || f == 1) k_fs_c2<N1, true><<<g2, kFsCols, G::SMEM, s>>>(a, fstw);
    if (f < 0 || f == 2) k_fs_inv_c1<N1><<<g1, kFsCols, G::SMEM, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_fs(int lg1, int lg2, bool inverse, const Dct2dArgs& a, const float2* fstw, int batch,
                   cudaStream_t s, bool prepare) {
#define GBDCT_FS_CASE(L1, L2, N1, N2) \
  if (lg1 == L1 && lg2 == L2) return fs_impl<N1, N2>(inverse, a, fstw, batch, s, prepare);
  GBDCT_FS_CASE(10, 12, 1024, 4096)
  GBDCT_FS_CASE(10, 13, 1024, 8192)
  GBDCT_FS_CASE(11, 12, 2048, 4096)
  GBDCT_FS_CASE(11, 13, 2048, 8192)
  GBDCT_FS_CASE(12, 12, 4096, 4096)
  GBDCT_FS_CASE(12, 13, 4096, 8192)
#undef GBDCT_FS_CASE
  return cudaErrorInvalidValue;
}

}  // namespace gbdct
