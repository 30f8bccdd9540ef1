// pass_fsp.cu - launches of the persistent pipelined four-step family.
#include "dct2d_launch.cuh"
#include "dct2d_pipe_kernels.cuh"

namespace gbdct {
namespace {

template <class Op>
cudaError_t pipe_launch(const Dct2dArgs& a, int nitems, int batch, int nsm, cudaStream_t s, bool prepare) {
  constexpr size_t smem = pipe_smem_bytes<Op>();
  if (prepare) {
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(k_pipe<Op>),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  const int grid = nitems < nsm ? nitems : nsm;
  k_pipe<Op><<<grid, kPipeThreads, smem, s>>>(a, batch);
  return cudaGetLastError();
}

template <int N1>
cudaError_t fsp_impl(bool inverse, const Dct2dArgs& a, int batch, int nsm, cudaStream_t s, bool prepare) {
  constexpr int N2 = 4096;
  using G = FsGeom<N1>;
  const int ncb = N2 / 2 / kFsCols;
  const int nA = G::A * ncb * batch, nB = G::B * ncb * batch, nR = (N1 / 4) * batch;
  cudaError_t e = cudaSuccess;
  if (prepare) {
    e = pipe_launch<FsColOp<N1, 0>>(a, 0, 0, 0, s, true);
    if (e == cudaSuccess) e = pipe_launch<FsColOp<N1, 1>>(a, 0, 0, 0, s, true);
    if (e == cudaSuccess) e = pipe_launch<FsColOp<N1, 2>>(a, 0, 0, 0, s, true);
    if (e == cudaSuccess) e = pipe_launch<FsColOp<N1, 3>>(a, 0, 0, 0, s, true);
    if (e == cudaSuccess) e = pipe_launch<FsRowOp<N1, N2, false>>(a, 0, 0, 0, s, true);
    if (e == cudaSuccess) e = pipe_launch<FsRowOp<N1, N2, true>>(a, 0, 0, 0, s, true);
    return e;
  }
  const int f = a.step_filter;
  if (!inverse) {
    if (f < 0 || f == 0) e = pipe_launch<FsColOp<N1, 0>>(a, nA, batch, nsm, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = pipe_launch<FsColOp<N1, 1>>(a, nB, batch, nsm, s, false);
    if (e == cudaSuccess && (f < 0 || f == 2))
      e = pipe_launch<FsRowOp<N1, N2, false>>(a, nR, batch, nsm, s, false);
  } else {
    if (f < 0 || f == 0) e = pipe_launch<FsRowOp<N1, N2, true>>(a, nR, batch, nsm, s, false);
    if (e == cudaSuccess && (f < 0 || f == 1)) e = pipe_launch<FsColOp<N1, 2>>(a, nB, batch, nsm, s, false);
    if (e == cudaSuccess && (f < 0 || f == 2)) e = pipe_launch<FsColOp<N1, 3>>(a, nA, batch, nsm, s, false);
  }
  return e;
}

}  // namespace

cudaError_t run_fsp(int lg1, int lg2, bool inverse, const Dct2dArgs& a, int batch, int nsm, cudaStream_t s,
                    bool prepare) {
  if (lg2 != 12) return cudaErrorInvalidValue;
  switch (lg1) {
    case 10: return fsp_impl<1024>(inverse, a, batch, nsm, s, prepare);
    case 11: return fsp_impl<2048>(inverse, a, batch, nsm, s, prepare);
    case 12: return fsp_impl<4096>(inverse, a, batch, nsm, s, prepare);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gbdct
