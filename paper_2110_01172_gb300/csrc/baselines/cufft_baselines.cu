// cufft_baselines.cu - comparison baselines, built into their own library
// (libgbdct_baselines.so); the transform library never uses them.
//
// B1, "DCT2D via RFFT2D" (Section III-C, Table V): the paper's own three-stage
// design with a library FFT.  Forward: a reorder kernel (Eq. 2d_dct_pre), the
// cuFFT 2D R2C transform, and a twiddle / symmetric-pair combine kernel whose
// thread writes the four outputs (k1,k2), (N1-k1,k2), (k1,N2-k2),
// (N1-k1,N2-k2) (Eqs. four-elements, s-t, with the 1/2 and periodic-index
// reading).  Inverse: the four-read preprocess (Eq. 2d_idct_pre, conjugate
// twiddles, 1/(N1 N2)), cuFFT 2D C2R, the inverse reorder (Eq. 2d_idct_post).
//
// B2, row-column (Section IV-A): the 1D DCT-II along the rows (row reorder,
// batched 1D cuFFT R2C, 1D twiddle X[k] = Re(e^{-i pi k / 2N} V[k]) written
// transposed through a shared-memory tile, with the next axis' reorder folded
// into the store), then the same along the other axis, transposed back.
// Forward only.
//
// FP32 arithmetic; twiddle tables from FP64.  Every entry returns 0 on
// success, a nonzero CUDA or cuFFT status otherwise.
#include <cuda_runtime.h>
#include <cufft.h>

#include <new>

namespace {

__device__ __forceinline__ int sigma(int n, int N) { return (n <= (N - 1) / 2) ? 2 * n : 2 * N - 2 * n - 1; }
__device__ __forceinline__ int sigma_inv(int r, int N) { return (r & 1) ? N - 1 - (r >> 1) : (r >> 1); }
__device__ __forceinline__ float2 cm(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cj(float2 a) { return make_float2(a.x, -a.y); }

// w[k] = exp(-i pi k / (2 N)), k < n (FP64, rounded once)
__global__ void k_tw(float2* w, int N, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi((double)k / (2.0 * N), &s, &c);
  w[k] = make_float2((float)c, (float)(-s));
}

// ---------------------------------------------------------------- B1 kernels
// Reorder (Eq. 2d_dct_pre): thread m of row r reads the adjacent pair
// x[sigma1(r)][2m, 2m+1] as one float2 and stores v[r][m] = x[.][2m] and
// v[r][N2-1-m] = x[.][2m+1] (both runs coalesced across the warp).
__global__ void k_b1_pre(const float* __restrict__ x, float* __restrict__ v, int n1, int n2) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (m >= n2 / 2) return;
  const float2 p = reinterpret_cast<const float2*>(x + (long long)sigma(r, n1) * n2)[m];
  float* vr = v + (long long)r * n2;
  vr[m] = p.x;
  vr[n2 - 1 - m] = p.y;
}

__global__ void k_b1_post(const float2* __restrict__ V, float* __restrict__ X, const float2* __restrict__ a,
                          const float2* __restrict__ b, int n1, int n2) {
  const int k2 = blockIdx.x * blockDim.x + threadIdx.x, k1 = blockIdx.y;  // k1 <= n1/2, k2 <= n2/2
  if (k2 > n2 / 2) return;
  const int H = n2 / 2 + 1;
  const int m1 = (n1 - k1) % n1;
  const float2 P = V[(long long)k1 * H + k2], Q = V[(long long)m1 * H + k2];
  const float2 av = a[k1], bv = b[k2];
  const float2 aP = cm(av, P), aQ = cm(cj(av), Q);
  const float2 s = cm(bv, make_float2(aP.x + aQ.x, aP.y + aQ.y));
  const float2 t = cm(bv, make_float2(aP.x - aQ.x, aP.y - aQ.y));
  const bool r2 = k1 != 0 && 2 * k1 != n1, c2 = k2 != 0 && 2 * k2 != n2;
  X[(long long)k1 * n2 + k2] = 0.5f * s.x;
  if (r2) X[(long long)(n1 - k1) * n2 + k2] = -0.5f * t.y;
  if (c2) X[(long long)k1 * n2 + (n2 - k2)] = -0.5f * s.y;
  if (r2 && c2) X[(long long)(n1 - k1) * n2 + (n2 - k2)] = -0.5f * t.x;
}

__global__ void k_b1_ipre(const float* __restrict__ C, float2* __restrict__ V, const float2* __restrict__ a,
                          const float2* __restrict__ b, int n1, int n2) {
  const int k2 = blockIdx.x * blockDim.x + threadIdx.x, k1 = blockIdx.y;
  if (k2 > n2 / 2) return;
  const float c1 = C[(long long)k1 * n2 + k2];
  const float c2 = (k1 && k2) ? C[(long long)(n1 - k1) * n2 + (n2 - k2)] : 0.f;
  const float c3 = k1 ? C[(long long)(n1 - k1) * n2 + k2] : 0.f;
  const float c4 = k2 ? C[(long long)k1 * n2 + (n2 - k2)] : 0.f;
  const float sc = 1.0f / ((float)n1 * (float)n2);
  const float2 w = cm(cj(a[k1]), cj(b[k2]));
  const float2 z = cm(w, make_float2(c1 - c2, -(c3 + c4)));
  V[(long long)k1 * (n2 / 2 + 1) + k2] = make_float2(sc * z.x, sc * z.y);
}

// Inverse reorder (Eq. 2d_idct_post), the mirror of k_b1_pre: one float2 store
// of x[sigma1(r)][2m, 2m+1] = (v[r][m], v[r][N2-1-m]) per thread.
__global__ void k_b1_ipost(const float* __restrict__ v, float* __restrict__ x, int n1, int n2) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (m >= n2 / 2) return;
  const float* vr = v + (long long)r * n2;
  reinterpret_cast<float2*>(x + (long long)sigma(r, n1) * n2)[m] = make_float2(vr[m], vr[n2 - 1 - m]);
}

// ---------------------------------------------------------------- B2 kernels
__global__ void k_b2_rowpre(const float* __restrict__ x, float* __restrict__ v, int rows, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (c >= n || r >= rows) return;
  v[(long long)r * n + c] = x[(long long)r * n + sigma(c, n)];
}

// W: rows x (n/2 + 1) half spectra of length-n rows.  Writes
// Y[k][dst(r)] = Re(e^{-i pi k / 2n} W(r, k)) for k < n (Hermitian mirror for
// k > n/2): the 1D DCT-II of row r, transposed, with dst = the reorder of
// the next axis (identity when last).  32 x 32 tiles through shared memory.
__global__ void k_b2_post_t(const float2* __restrict__ W, float* __restrict__ Y, const float2* __restrict__ w,
                            int rows, int n, int reorder_rows) {
  __shared__ float tile[32][33];
  const int H = n / 2 + 1;
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, k = k0 + threadIdx.x;
    float val = 0.f;
    if (r < rows && k < n) {
      const float2 z = (k <= n / 2) ? W[(long long)r * H + k] : cj(W[(long long)r * H + (n - k)]);
      const float2 tw = w[k];
      val = tw.x * z.x - tw.y * z.y;
    }
    tile[i][threadIdx.x] = val;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, r = r0 + threadIdx.x;
    if (k < n && r < rows) {
      const int d = reorder_rows ? sigma_inv(r, rows) : r;
      Y[(long long)k * rows + d] = tile[threadIdx.x][i];
    }
  }
}

}  // namespace

struct gbdct_b1_s {
  int n1, n2;
  cufftHandle r2c, c2r;
  bool has_r2c = false, has_c2r = false;
  float* v;
  float2* V;
  float2 *a, *b;  // a: n1 entries, b: n2 entries
};

struct gbdct_b2_s {
  int n1, n2;
  cufftHandle rows1, rows2;  // batched 1D R2C: n1 rows of n2, then n2 rows of n1
  bool has_rows1 = false, has_rows2 = false;
  float *v, *y;
  float2* W;
  float2 *a, *b;
};

extern "C" {

int gbdct_b1_destroy(gbdct_b1_s* p);
int gbdct_b2_destroy(gbdct_b2_s* p);

int gbdct_b1_create(gbdct_b1_s** out, int n1, int n2) {
  gbdct_b1_s* p = new (std::nothrow) gbdct_b1_s();
  if (!p) return -1;
  p->n1 = n1;
  p->n2 = n2;
  int st = cufftPlan2d(&p->r2c, n1, n2, CUFFT_R2C);
  p->has_r2c = !st;
  if (!st) {
    st = cufftPlan2d(&p->c2r, n1, n2, CUFFT_C2R);
    p->has_c2r = !st;
  }
  cudaError_t e = cudaSuccess;
  if (!st) e = cudaMalloc(&p->v, sizeof(float) * n1 * n2);
  if (!st && !e) e = cudaMalloc(&p->V, sizeof(float2) * n1 * (n2 / 2 + 1));
  if (!st && !e) e = cudaMalloc(&p->a, sizeof(float2) * n1);
  if (!st && !e) e = cudaMalloc(&p->b, sizeof(float2) * n2);
  if (!st && !e) {
    k_tw<<<(n1 + 255) / 256, 256>>>(p->a, n1, n1);
    k_tw<<<(n2 + 255) / 256, 256>>>(p->b, n2, n2);
    e = cudaDeviceSynchronize();
  }
  if (st || e) {
    gbdct_b1_destroy(p);
    *out = nullptr;
    return st ? st : (int)e;
  }
  *out = p;
  return 0;
}

int gbdct_b1_forward(gbdct_b1_s* p, const float* x, float* X, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n1 = p->n1, n2 = p->n2;
  k_b1_pre<<<dim3((n2 / 2 + 255) / 256, n1), 256, 0, s>>>(x, p->v, n1, n2);
  int st = cufftSetStream(p->r2c, s);
  if (!st) st = cufftExecR2C(p->r2c, p->v, reinterpret_cast<cufftComplex*>(p->V));
  k_b1_post<<<dim3((n2 / 2 + 1 + 255) / 256, n1 / 2 + 1), 256, 0, s>>>(p->V, X, p->a, p->b, n1, n2);
  return st ? st : (int)cudaGetLastError();
}

int gbdct_b1_inverse(gbdct_b1_s* p, const float* C, float* x, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n1 = p->n1, n2 = p->n2;
  k_b1_ipre<<<dim3((n2 / 2 + 1 + 255) / 256, n1), 256, 0, s>>>(C, p->V, p->a, p->b, n1, n2);
  int st = cufftSetStream(p->c2r, s);
  if (!st) st = cufftExecC2R(p->c2r, reinterpret_cast<cufftComplex*>(p->V), p->v);
  k_b1_ipost<<<dim3((n2 / 2 + 255) / 256, n1), 256, 0, s>>>(p->v, x, n1, n2);
  return st ? st : (int)cudaGetLastError();
}

// The library FFTs of B1 alone (the paper's "RFFT2D" / "IRFFT2D" columns of
// Table V): cuFFT 2D R2C of the plan's real buffer and C2R back into it.
int gbdct_b1_r2c_only(gbdct_b1_s* p, void* stream) {
  int st = cufftSetStream(p->r2c, reinterpret_cast<cudaStream_t>(stream));
  if (!st) st = cufftExecR2C(p->r2c, p->v, reinterpret_cast<cufftComplex*>(p->V));
  return st;
}

int gbdct_b1_c2r_only(gbdct_b1_s* p, void* stream) {
  int st = cufftSetStream(p->c2r, reinterpret_cast<cudaStream_t>(stream));
  if (!st) st = cufftExecC2R(p->c2r, reinterpret_cast<cufftComplex*>(p->V), p->v);
  return st;
}

int gbdct_b1_destroy(gbdct_b1_s* p) {
  if (!p) return 0;
  if (p->has_r2c) cufftDestroy(p->r2c);
  if (p->has_c2r) cufftDestroy(p->c2r);
  cudaFree(p->v);
  cudaFree(p->V);
  cudaFree(p->a);
  cudaFree(p->b);
  delete p;
  return 0;
}

int gbdct_b2_create(gbdct_b2_s** out, int n1, int n2) {
  gbdct_b2_s* p = new (std::nothrow) gbdct_b2_s();
  if (!p) return -1;
  p->n1 = n1;
  p->n2 = n2;
  int len2 = n2, len1 = n1;
  int st = cufftPlanMany(&p->rows1, 1, &len2, nullptr, 1, n2, nullptr, 1, n2 / 2 + 1, CUFFT_R2C, n1);
  p->has_rows1 = !st;
  if (!st) {
    st = cufftPlanMany(&p->rows2, 1, &len1, nullptr, 1, n1, nullptr, 1, n1 / 2 + 1, CUFFT_R2C, n2);
    p->has_rows2 = !st;
  }
  cudaError_t e = cudaSuccess;
  const size_t hw = (size_t)n1 * (n2 / 2 + 1) > (size_t)n2 * (n1 / 2 + 1) ? (size_t)n1 * (n2 / 2 + 1)
                                                                            : (size_t)n2 * (n1 / 2 + 1);
  if (!st) e = cudaMalloc(&p->v, sizeof(float) * n1 * n2);
  if (!st && !e) e = cudaMalloc(&p->y, sizeof(float) * n1 * n2);
  if (!st && !e) e = cudaMalloc(&p->W, sizeof(float2) * hw);
  if (!st && !e) e = cudaMalloc(&p->a, sizeof(float2) * n1);
  if (!st && !e) e = cudaMalloc(&p->b, sizeof(float2) * n2);
  if (!st && !e) {
    k_tw<<<(n1 + 255) / 256, 256>>>(p->a, n1, n1);
    k_tw<<<(n2 + 255) / 256, 256>>>(p->b, n2, n2);
    e = cudaDeviceSynchronize();
  }
  if (st || e) {
    gbdct_b2_destroy(p);
    *out = nullptr;
    return st ? st : (int)e;
  }
  *out = p;
  return 0;
}

int gbdct_b2_forward(gbdct_b2_s* p, const float* x, float* X, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n1 = p->n1, n2 = p->n2;
  const dim3 tb(32, 8);
  // axis 1 (rows of length n2): reorder, R2C, twiddle + transpose to (n2, n1)
  // with the axis-0 reorder folded into the store
  k_b2_rowpre<<<dim3((n2 + 255) / 256, n1), 256, 0, s>>>(x, p->v, n1, n2);
  int st = cufftSetStream(p->rows1, s);
  if (!st) st = cufftExecR2C(p->rows1, p->v, reinterpret_cast<cufftComplex*>(p->W));
  k_b2_post_t<<<dim3((n2 + 31) / 32, (n1 + 31) / 32), tb, 0, s>>>(p->W, p->y, p->b, n1, n2, 1);
  // axis 0 (rows of length n1 of the transposed array): R2C, twiddle + transpose back
  if (!st) st = cufftSetStream(p->rows2, s);
  if (!st) st = cufftExecR2C(p->rows2, p->y, reinterpret_cast<cufftComplex*>(p->W));
  k_b2_post_t<<<dim3((n1 + 31) / 32, (n2 + 31) / 32), tb, 0, s>>>(p->W, X, p->a, n2, n1, 0);
  return st ? st : (int)cudaGetLastError();
}

int gbdct_b2_destroy(gbdct_b2_s* p) {
  if (!p) return 0;
  if (p->has_rows1) cufftDestroy(p->rows1);
  if (p->has_rows2) cufftDestroy(p->rows2);
  cudaFree(p->v);
  cudaFree(p->y);
  cudaFree(p->W);
  cudaFree(p->a);
  cudaFree(p->b);
  delete p;
  return 0;
}

}  // extern "C"
