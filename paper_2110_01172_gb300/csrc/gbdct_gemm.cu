// gbdct_gemm.cu - split-BF16 DFT-GEMM precision mode (see gemm_path.cuh): the
// two dense products of the separable definition on the tensor cores, by the
// hand-written tcgen05 kernel of tc_gemm.cuh.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>
#include <new>

#include "gemm_path.cuh"
#include "tc_gemm.cuh"

namespace gbdct {

struct GemmPath {
  int n1 = 0, n2 = 0, batch = 0, nsm = 0;
  int* err = nullptr;                          // the plan's device error word
  uint32_t polls = tc::kDefaultPolls;          // bound of every device-side wait
  // row-major N x N matrices, split: C1h C1l D1h D1l (n1), C2h C2l D2h D2l (n2)
  __nv_bfloat16* mats = nullptr;
  __nv_bfloat16 *xh = nullptr, *xl = nullptr;  // split input, [batch n1][n2]
  __nv_bfloat16 *th = nullptr, *tl = nullptr;  // split intermediate, transposed: [batch n2][n1]
  size_t bytes = 0;
  // tensor maps (box 64 x 128 for A operands; 64 x 128 and 64 x 64 for B operands)
  CUtensorMap xa[2];           // x hi / lo as A of the first product
  CUtensorMap ra[2][4];        // [BN 128 / 64][C2h, C2l, D2h, D2l] as B of the first product
  CUtensorMap la[4];           // C1h, C1l, D1h, D1l as A of the second product
  CUtensorMap tb[2][2];        // [BN 128 / 64][T hi, T lo] as B of the second product
};

namespace {

// Matrix entry in FP64 from the integer-reduced angle m = k (2j+1) mod 4N.
__device__ double cos_half(long long m, int n) { return cospi((double)(m % (4LL * n)) / (2.0 * n)); }

// C (DCT-II, rows index the output) and D = (2/N) C^T diag(w) for one side n,
// split into bf16 hi / lo.
__global__ void k_gemm_mats(__nv_bfloat16* ch, __nv_bfloat16* cl, __nv_bfloat16* dh, __nv_bfloat16* dl, int n) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int r = (int)(idx / n), c = (int)(idx % n);
  const double cv = cos_half((long long)r * (2 * c + 1), n);                                 // C[r][c]
  const double dv = (2.0 / n) * (c ? 1.0 : 0.5) * cos_half((long long)c * (2 * r + 1), n);  // D[r][c]
  const __nv_bfloat16 chv = __float2bfloat16_rn((float)cv), dhv = __float2bfloat16_rn((float)dv);
  ch[idx] = chv;
  cl[idx] = __float2bfloat16_rn((float)(cv - (double)__bfloat162float(chv)));
  dh[idx] = dhv;
  dl[idx] = __float2bfloat16_rn((float)(dv - (double)__bfloat162float(dhv)));
}

__global__ void k_split(const float* __restrict__ v, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                        long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = v[i];
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  hi[i] = h;
  lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() { return tma::encoder(); }

// 2D bf16 map of a row-major rows x cols matrix, box 64 (cols) x box_rows, 128-byte swizzle.
bool map2d(CUtensorMap* m, const void* base, long long rows, long long cols, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                   const tc::Epi& e, int rows, int cols, int kdim, int nz, uint32_t polls, int* err, cudaStream_t s) {
  using Cf = tc::Cfg<BN>;
  const dim3 grid((unsigned)(cols / BN), (unsigned)(rows / tc::BM), (unsigned)nz);
  tc::k_tc_dftgemm<BN><<<grid, 128, Cf::SMEM, s>>>(ah, al, bh, bl, e, kdim / tc::BK, polls, err);
  return cudaGetLastError();
}

// BN = 128 when that already gives at least one tile per SM, else 64.
bool wide_tiles(long long rows, long long cols, int nz, int nsm) {
  return (rows / tc::BM) * (cols / 128) * nz >= nsm;
}

}  // namespace

GemmPath* gemm_create(int n1, int n2, int batch, int* err, gbdct_status* st) {
  *st = GBDCT_ERR_UNSUPPORTED;
  if (n1 < kGemmMinSide || n2 < kGemmMinSide || n1 > kGemmMaxSide || n2 > kGemmMaxSide || batch < 1) return nullptr;
  GemmPath* g = new (std::nothrow) GemmPath();
  if (!g) {
    *st = GBDCT_ERR_OOM;
    return nullptr;
  }
  g->n1 = n1;
  g->n2 = n2;
  g->batch = batch;
  g->err = err;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&g->nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t m1 = (size_t)n1 * n1, m2 = (size_t)n2 * n2, e = (size_t)batch * n1 * n2;
  if (ce == cudaSuccess) ce = cudaMalloc(&g->mats, (4 * m1 + 4 * m2) * sizeof(__nv_bfloat16));
  if (ce == cudaSuccess) ce = cudaMalloc(&g->xh, 4 * e * sizeof(__nv_bfloat16));  // xh, xl, th, tl
  g->bytes = (4 * m1 + 4 * m2) * sizeof(__nv_bfloat16) + 4 * e * sizeof(__nv_bfloat16);
  if (ce == cudaSuccess) {
    g->xl = g->xh + e;
    g->th = g->xl + e;
    g->tl = g->th + e;
    __nv_bfloat16* m = g->mats;
    k_gemm_mats<<<(unsigned)((m1 + 255) / 256), 256>>>(m, m + m1, m + 2 * m1, m + 3 * m1, n1);
    __nv_bfloat16* q = m + 4 * m1;
    k_gemm_mats<<<(unsigned)((m2 + 255) / 256), 256>>>(q, q + m2, q + 2 * m2, q + 3 * m2, n2);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  }
  if (ce == cudaSuccess) ce = cudaFuncSetAttribute(reinterpret_cast<const void*>(tc::k_tc_dftgemm<128>),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Cfg<128>::SMEM);
  if (ce == cudaSuccess) ce = cudaFuncSetAttribute(reinterpret_cast<const void*>(tc::k_tc_dftgemm<64>),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Cfg<64>::SMEM);
  bool maps = ce == cudaSuccess;
  if (maps) {
    const __nv_bfloat16* m = g->mats;
    const __nv_bfloat16* q = m + 4 * m1;
    const long long rows1 = (long long)batch * n1;
    maps = map2d(&g->xa[0], g->xh, rows1, n2, tc::BM) && map2d(&g->xa[1], g->xl, rows1, n2, tc::BM);
    for (int w = 0; w < 2 && maps; ++w) {
      const int bn = w ? 64 : 128;
      for (int i = 0; i < 4 && maps; ++i) maps = map2d(&g->ra[w][i], q + i * m2, n2, n2, bn);
      maps = maps && map2d(&g->tb[w][0], g->th, (long long)batch * n2, n1, bn) &&
             map2d(&g->tb[w][1], g->tl, (long long)batch * n2, n1, bn);
    }
    for (int i = 0; i < 4 && maps; ++i) maps = map2d(&g->la[i], m + i * m1, n1, n1, tc::BM);
  }
  if (ce != cudaSuccess || !maps) {
    gemm_destroy(g);
    *st = ce == cudaErrorMemoryAllocation ? GBDCT_ERR_OOM : GBDCT_ERR_CUDA;
    return nullptr;
  }
  *st = GBDCT_OK;
  return g;
}

void gemm_set_wait_polls(GemmPath* g, uint32_t polls) {
  if (g) g->polls = polls ? polls : tc::kDefaultPolls;
}

gbdct_status gemm_exec(GemmPath* g, bool inverse, const float* in, float* out, cudaStream_t s) {
  const int n1 = g->n1, n2 = g->n2;
  const long long e = (long long)g->batch * n1 * n2;
  const int r0 = inverse ? 2 : 0;  // forward: C1, C2; inverse: D1, D2
  k_split<<<(unsigned)((e + 255) / 256), 256, 0, s>>>(in, g->xh, g->xl, e);
  cudaError_t ce = cudaGetLastError();
  // first product T = x R^T (rows: batch * n1), stored split and transposed
  tc::Epi e1{tc::EPI_SPLIT_T, n1, n2, 0, 0, g->th, g->tl, nullptr};
  const long long rows1 = (long long)g->batch * n1;
  if (ce == cudaSuccess) {
    const bool wide = wide_tiles(rows1, n2, 1, g->nsm);
    ce = wide ? launch<128>(g->xa[0], g->xa[1], g->ra[0][r0], g->ra[0][r0 + 1], e1, (int)rows1, n2, n2, 1, g->polls,
                            g->err, s)
              : launch<64>(g->xa[0], g->xa[1], g->ra[1][r0], g->ra[1][r0 + 1], e1, (int)rows1, n2, n2, 1, g->polls,
                           g->err, s);
  }
  // second product out_b = L T_b (rows n1 per batch entry)
  tc::Epi e2{tc::EPI_F32, n1, n2, 0, n2, nullptr, nullptr, out};
  if (ce == cudaSuccess) {
    const bool wide = wide_tiles(n1, n2, g->batch, g->nsm);
    ce = wide ? launch<128>(g->la[r0], g->la[r0 + 1], g->tb[0][0], g->tb[0][1], e2, n1, n2, n1, g->batch, g->polls,
                            g->err, s)
              : launch<64>(g->la[r0], g->la[r0 + 1], g->tb[1][0], g->tb[1][1], e2, n1, n2, n1, g->batch, g->polls,
                           g->err, s);
  }
  return ce == cudaSuccess ? GBDCT_OK : GBDCT_ERR_CUDA;
}

size_t gemm_workspace_bytes(const GemmPath* g) { return g ? g->bytes : 0; }

void gemm_destroy(GemmPath* g) {
  if (!g) return;
  cudaFree(g->mats);
  cudaFree(g->xh);
  delete g;
}

}  // namespace gbdct
