// gbdct_gemm.cu - split-BF16 DFT-GEMM precision mode (see gemm_path.cuh).
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <new>

#include "gemm_path.cuh"

namespace gbdct {

struct GemmPath {
  int n1 = 0, n2 = 0, batch = 0;
  cublasHandle_t h = nullptr;
  // row-major N x N matrices, split: [C1 hi, C1 lo, C2 hi, C2 lo, D1 hi, D1 lo, D2 hi, D2 lo]
  __nv_bfloat16* mats = nullptr;
  __nv_bfloat16 *ah = nullptr, *al = nullptr;  // split operand (x, then the intermediate)
  float* t = nullptr;                          // FP32 intermediate
  size_t bytes = 0;
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

gbdct_status blas(cublasStatus_t s) { return s == CUBLAS_STATUS_SUCCESS ? GBDCT_OK : GBDCT_ERR_CUDA; }

// out (rows x n2, row-major, FP32) = A (rows x n2) * M^T (M: n2 x n2, row-major)
// with the split products hi hi + hi lo + lo hi.
gbdct_status right_product(GemmPath* g, const __nv_bfloat16* Ah, const __nv_bfloat16* Al, const __nv_bfloat16* Mh,
                           const __nv_bfloat16* Ml, float* out, int rows, int n2) {
  const float one = 1.f, zero = 0.f;
  const __nv_bfloat16* ms[3] = {Mh, Ml, Mh};
  const __nv_bfloat16* as[3] = {Ah, Ah, Al};
  for (int i = 0; i < 3; ++i) {
    // column-major view: out^T (n2 x rows) = M (op T of the stored M^T) * A^T
    const gbdct_status st = blas(cublasGemmEx(g->h, CUBLAS_OP_T, CUBLAS_OP_N, n2, rows, n2, &one, ms[i], CUDA_R_16BF,
                                              n2, as[i], CUDA_R_16BF, n2, i ? &one : &zero, out, CUDA_R_32F, n2,
                                              CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT));
    if (st != GBDCT_OK) return st;
  }
  return GBDCT_OK;
}

// out_b (n1 x n2) = L (n1 x n1, row-major) * T_b (n1 x n2), for every batch entry b.
gbdct_status left_product(GemmPath* g, const __nv_bfloat16* Th, const __nv_bfloat16* Tl, const __nv_bfloat16* Lh,
                          const __nv_bfloat16* Ll, float* out) {
  const int n1 = g->n1, n2 = g->n2;
  const long long st_t = (long long)n1 * n2;
  const float one = 1.f, zero = 0.f;
  const __nv_bfloat16* ts[3] = {Th, Tl, Th};
  const __nv_bfloat16* ls[3] = {Lh, Lh, Ll};
  for (int i = 0; i < 3; ++i) {
    // column-major view: out_b^T (n2 x n1) = T_b^T (n2 x n1) * L^T (n1 x n1)
    const gbdct_status st = blas(cublasGemmStridedBatchedEx(
        g->h, CUBLAS_OP_N, CUBLAS_OP_N, n2, n1, n1, &one, ts[i], CUDA_R_16BF, n2, st_t, ls[i], CUDA_R_16BF, n1, 0,
        i ? &one : &zero, out, CUDA_R_32F, n2, st_t, g->batch, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT));
    if (st != GBDCT_OK) return st;
  }
  return GBDCT_OK;
}

}  // namespace

GemmPath* gemm_create(int n1, int n2, int batch, gbdct_status* st) {
  *st = GBDCT_ERR_UNSUPPORTED;
  if (n1 < 2 || n2 < 2 || n1 > kGemmMaxSide || n2 > kGemmMaxSide || batch < 1) return nullptr;
  GemmPath* g = new (std::nothrow) GemmPath();
  if (!g) {
    *st = GBDCT_ERR_OOM;
    return nullptr;
  }
  g->n1 = n1;
  g->n2 = n2;
  g->batch = batch;
  const size_t m1 = (size_t)n1 * n1, m2 = (size_t)n2 * n2, e = (size_t)batch * n1 * n2;
  cudaError_t ce = cudaMalloc(&g->mats, (4 * m1 + 4 * m2) * sizeof(__nv_bfloat16));
  if (ce == cudaSuccess) ce = cudaMalloc(&g->ah, e * sizeof(__nv_bfloat16));
  if (ce == cudaSuccess) ce = cudaMalloc(&g->al, e * sizeof(__nv_bfloat16));
  if (ce == cudaSuccess) ce = cudaMalloc(&g->t, e * sizeof(float));
  g->bytes = (4 * m1 + 4 * m2) * sizeof(__nv_bfloat16) + 2 * e * sizeof(__nv_bfloat16) + e * sizeof(float);
  if (ce == cudaSuccess) {
    __nv_bfloat16* m = g->mats;
    // layout: C1h C1l D1h D1l (n1), C2h C2l D2h D2l (n2)
    k_gemm_mats<<<(unsigned)((m1 + 255) / 256), 256>>>(m, m + m1, m + 2 * m1, m + 3 * m1, n1);
    __nv_bfloat16* q = m + 4 * m1;
    k_gemm_mats<<<(unsigned)((m2 + 255) / 256), 256>>>(q, q + m2, q + 2 * m2, q + 3 * m2, n2);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  }
  if (ce != cudaSuccess) {
    gemm_destroy(g);
    *st = ce == cudaErrorMemoryAllocation ? GBDCT_ERR_OOM : GBDCT_ERR_CUDA;
    return nullptr;
  }
  if (cublasCreate(&g->h) != CUBLAS_STATUS_SUCCESS) {
    g->h = nullptr;
    gemm_destroy(g);
    *st = GBDCT_ERR_CUDA;
    return nullptr;
  }
  *st = GBDCT_OK;
  return g;
}

gbdct_status gemm_exec(GemmPath* g, bool inverse, const float* in, float* out, cudaStream_t s) {
  const int n1 = g->n1, n2 = g->n2;
  const size_t m1 = (size_t)n1 * n1, m2 = (size_t)n2 * n2;
  const long long e = (long long)g->batch * n1 * n2;
  const __nv_bfloat16* m = g->mats;
  const __nv_bfloat16* q = m + 4 * m1;
  // forward: L = C1, R = C2; inverse: L = D1, R = D2
  const __nv_bfloat16 *Lh = m + (inverse ? 2 * m1 : 0), *Ll = Lh + m1;
  const __nv_bfloat16 *Rh = q + (inverse ? 2 * m2 : 0), *Rl = Rh + m2;
  if (cublasSetStream(g->h, s) != CUBLAS_STATUS_SUCCESS) return GBDCT_ERR_CUDA;
  const unsigned blocks = (unsigned)((e + 255) / 256);
  k_split<<<blocks, 256, 0, s>>>(in, g->ah, g->al, e);
  if (cudaGetLastError() != cudaSuccess) return GBDCT_ERR_CUDA;
  gbdct_status st = right_product(g, g->ah, g->al, Rh, Rl, g->t, g->batch * n1, n2);  // T = in R^T
  if (st != GBDCT_OK) return st;
  k_split<<<blocks, 256, 0, s>>>(g->t, g->ah, g->al, e);
  if (cudaGetLastError() != cudaSuccess) return GBDCT_ERR_CUDA;
  return left_product(g, g->ah, g->al, Lh, Ll, out);  // out_b = L T_b
}

size_t gemm_workspace_bytes(const GemmPath* g) { return g ? g->bytes : 0; }

void gemm_destroy(GemmPath* g) {
  if (!g) return;
  if (g->h) cublasDestroy(g->h);
  cudaFree(g->mats);
  cudaFree(g->ah);
  cudaFree(g->al);
  cudaFree(g->t);
  delete g;
}

}  // namespace gbdct
