// gbdct_poisson.cu - spectral Neumann Poisson solve (Section V-B, Algorithm 4).
//
// density rho -> a = DCT-II(rho) -> potential psi = IDCT(a / (wu^2 + wv^2)),
// field xi0 = IDXST_IDCT(a wu / (wu^2 + wv^2)), xi1 = IDCT_IDXST(a wv / (...)),
// with wu = pi u / N1, wv = pi v / N2 and the DC term zeroed (the paper's
// "scaled electric potential a1, a2"; the scaling is the grid-unit
// eigenfrequency reading of the cosine basis).  The transforms are the
// library's own plans; one kernel applies the three spectral scalings.
// The eigenvalue denominators 1 / (wu^2 + wv^2) are evaluated in FP64 once,
// when the solver is created, and rounded once into an FP32 table that every
// solve reads; wu and wv are FP64 values rounded once as well.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "../../include/gbdct.h"

struct gbdct_poisson_s {
  int n1, n2, device;
  gbdct_plan_t fwd, fld0, fld1;  // DCT2 (forward and potential inverse), IDXST_IDCT, IDCT_IDXST
  float* w;    // wu[N1], wv[N2]
  float* inv;  // 1 / (wu^2 + wv^2) per (u, v), 0 at (0, 0): N1 x N2
};

namespace {

// Eigenfrequency tables in FP64, rounded once: wu = pi u / N1, wv = pi v / N2.
__global__ void k_poisson_tables(float* w, int n1, int n2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) w[i] = (float)(3.14159265358979323846 * (double)i / (double)n1);
  if (i < n2) w[n1 + i] = (float)(3.14159265358979323846 * (double)i / (double)n2);
}

// Eigenvalue denominators in FP64, rounded once: inv(u, v) = 1 / (wu^2 + wv^2),
// inv(0, 0) = 0 (the DC term is zeroed).
__global__ void k_poisson_denominators(float* inv, int n1, int n2) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  if (v >= n2) return;
  const double wu = 3.14159265358979323846 * (double)u / (double)n1;
  const double wv = 3.14159265358979323846 * (double)v / (double)n2;
  inv[(long long)u * n2 + v] = (u | v) ? (float)(1.0 / (wu * wu + wv * wv)) : 0.0f;
}

// In place on `a` (becomes a / den), and writes a wu / den, a wv / den.
__global__ void k_poisson_scale(float* __restrict__ a, float* __restrict__ a1, float* __restrict__ a2,
                                const float* __restrict__ w, const float* __restrict__ inv, int n1, int n2) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  if (v >= n2) return;
  const float wu = __ldg(w + u), wv = __ldg(w + n1 + v);
  const long long idx = (long long)u * n2 + v;
  const float val = a[idx] * __ldg(inv + idx);
  a[idx] = val;
  a1[idx] = val * wu;
  a2[idx] = val * wv;
}

// Makes the solver's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

void destroy(gbdct_poisson_s* p) {
  if (!p) return;
  gbdct_plan_destroy(p->fwd);
  gbdct_plan_destroy(p->fld0);
  gbdct_plan_destroy(p->fld1);
  if (p->w) cudaFree(p->w);
  if (p->inv) cudaFree(p->inv);
  delete p;
}

}  // namespace

extern "C" {

gbdct_status gbdct_poisson_create(gbdct_poisson_t* out, int64_t n1, int64_t n2) {
  if (!out) return GBDCT_ERR_INVALID_ARG;
  const int64_t dims[2] = {n1, n2};
  gbdct_poisson_s* p = new (std::nothrow) gbdct_poisson_s();
  if (!p) return GBDCT_ERR_OOM;
  gbdct_status st = gbdct_plan_create(&p->fwd, 2, dims, GBDCT_DCT2, GBDCT_F32);
  if (st == GBDCT_OK) st = gbdct_plan_create(&p->fld0, 2, dims, GBDCT_IDXST_IDCT, GBDCT_F32);
  if (st == GBDCT_OK) st = gbdct_plan_create(&p->fld1, 2, dims, GBDCT_IDCT_IDXST, GBDCT_F32);
  if (st != GBDCT_OK) {
    destroy(p);
    return st;
  }
  p->n1 = (int)n1;
  p->n2 = (int)n2;
  cudaGetDevice(&p->device);
  cudaError_t e = cudaMalloc(&p->w, (size_t)(n1 + n2) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&p->inv, (size_t)n1 * (size_t)n2 * sizeof(float));
  if (e == cudaSuccess) {
    const int m = (int)(n1 > n2 ? n1 : n2);
    k_poisson_tables<<<(m + 255) / 256, 256>>>(p->w, (int)n1, (int)n2);
    k_poisson_denominators<<<dim3((unsigned)((n2 + 255) / 256), (unsigned)n1), 256>>>(p->inv, (int)n1, (int)n2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    destroy(p);
    return e == cudaErrorMemoryAllocation ? GBDCT_ERR_OOM : GBDCT_ERR_CUDA;
  }
  *out = p;
  return GBDCT_OK;
}

gbdct_status gbdct_poisson_solve(gbdct_poisson_t p, const void* rho, void* psi, void* xi0, void* xi1,
                                 void* stream) {
  if (!p || !rho || !psi || !xi0 || !xi1) return GBDCT_ERR_INVALID_ARG;
  if (psi == xi0 || psi == xi1 || xi0 == xi1) return GBDCT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  gbdct_status st = gbdct_exec_forward(p->fwd, rho, psi, stream);
  if (st != GBDCT_OK) return st;
  const dim3 grid((p->n2 + 255) / 256, p->n1);
  k_poisson_scale<<<grid, 256, 0, s>>>(static_cast<float*>(psi), static_cast<float*>(xi0),
                                       static_cast<float*>(xi1), p->w, p->inv, p->n1, p->n2);
  if (cudaGetLastError() != cudaSuccess) return GBDCT_ERR_CUDA;
  st = gbdct_exec_inverse(p->fwd, psi, psi, stream);
  if (st == GBDCT_OK) st = gbdct_exec_inverse(p->fld0, xi0, xi0, stream);
  if (st == GBDCT_OK) st = gbdct_exec_inverse(p->fld1, xi1, xi1, stream);
  return st;
}

size_t gbdct_poisson_workspace_bytes(gbdct_poisson_t p) {
  if (!p) return 0;
  return gbdct_plan_workspace_bytes(p->fwd) + gbdct_plan_workspace_bytes(p->fld0) + gbdct_plan_workspace_bytes(p->fld1) +
         (size_t)p->n1 * p->n2 * sizeof(float) /* denominators */ + (size_t)(p->n1 + p->n2) * sizeof(float);
}

gbdct_status gbdct_poisson_destroy(gbdct_poisson_t p) {
  if (!p) return GBDCT_OK;
  DeviceGuard guard(p->device);
  destroy(p);
  return GBDCT_OK;
}

}  // extern "C"
