// gbdct_noalloc.cu - forward 2D DCT-II that allocates no device memory.
//
// For callers that must not allocate device memory on the call path: code
// running inside a host framework that owns all device memory through its
// own pool and forbids raw cudaMalloc, or latency-critical loops where a
// cudaMalloc/cudaFree (which may synchronise the device) would stall other
// work.  The workspace and twiddle tables live in a file-scope static
// __device__ array instead of plan-owned allocations; every call rebuilds the
// tables there and then runs the same two fused passes as
// gbdct_exec_forward.  Limits and set-up rules are documented in gbdct.h.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/gbdct.h"
#include "dct2d_launch.cuh"

namespace {

constexpr int64_t kNoAllocMaxElems = int64_t(1) << 20;           // N1 * N2 limit
constexpr size_t kWorkBytes = size_t(kNoAllocMaxElems) * 4;      // (N1/2) * N2 complex
constexpr size_t kTableElems = size_t(1) << 17;                  // float2, >= every table below
constexpr size_t kScratchBytes = kWorkBytes + kTableElems * sizeof(float2);

// The shared scratch: every call on a device uses (and overwrites) it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Stage twiddles of the 16-point-per-thread stage structure (fft_core.cuh):
// entry (j-1)*NS + k of the stage starting at NS is exp(-2 pi i j k/(NS R)).
__global__ void k_na_stage_twiddles(float2* out, int L, int total) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int off = 0;
  for (int ns = 1; ns < L; ns *= gbdct::stage_radix(L, ns)) {
    const int R = gbdct::stage_radix(L, ns);
    if (ns == 1) continue;
    const int sz = (R - 1) * ns;
    if (idx < off + sz) {
      const int e = idx - off;
      const long long j = e / ns + 1, k = e % ns, M = (long long)ns * R;
      double sn, cs;
      sincospi(-2.0 * (double)((j * k) % M) / (double)M, &sn, &cs);
      out[idx] = make_float2((float)cs, (float)sn);
      return;
    }
    off += sz;
  }
}

// a_k, b_k / 2 (forward combine of Section III-B); the inverse tables are
// not needed by the forward transform.
__global__ void k_na_dct_tables(float2* fa, float2* fb, int n1, int n2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx <= n1 / 2) {
    double sn, cs;
    sincospi((double)idx / (2.0 * (double)n1), &sn, &cs);
    fa[idx] = make_float2((float)cs, (float)(-sn));
  }
  if (idx < n2) {
    double sn, cs;
    sincospi((double)idx / (2.0 * (double)n2), &sn, &cs);
    fb[idx] = make_float2((float)(0.5 * cs), (float)(-0.5 * sn));
  }
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int lg2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}
size_t up2(size_t v) { return (v + 1) & ~size_t(1); }

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress needs that device current).
gbdct_status scratch_for_current_device(float2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBDCT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GBDCT_ERR_CUDA;
    // The forward passes launched below need more than 48 KB of dynamic shared
    // memory at the largest sizes; raise the limits once per device as well.
    gbdct::Dct2dArgs a{};
    for (int lg = gbdct::kPairMinLog2; lg <= gbdct::kPairMaxLog2; ++lg) {
      if (gbdct::run_fwd_cols2(lg, a, 1, 1, 0, true) != cudaSuccess ||
          gbdct::run_fwd_rows2(lg, a, 1, 1, 0, true) != cudaSuccess)
        return GBDCT_ERR_CUDA;
    }
    for (int lg = gbdct::kMinLog2; lg <= gbdct::kMaxLog2; ++lg) {
      const int L = 1 << lg;
      a.seq_per_cta = gbdct::choose_seq_per_cta(L, 1 << 13);
      if (gbdct::run_fwd_cols(lg, a, dim3(1), 0, true) != cudaSuccess ||
          gbdct::run_fwd_rows(lg, a, dim3(1), 0, true) != cudaSuccess)
        return GBDCT_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<float2*>(g_scratch_ptr[dev]);
  return GBDCT_OK;
}

}  // namespace

extern "C" gbdct_status gbdct_dct2d_forward_noalloc(const void* in, void* out, int64_t n1, int64_t n2,
                                                    void* stream) {
  if (!in || !out) return GBDCT_ERR_INVALID_ARG;
  if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u)) return GBDCT_ERR_INVALID_ARG;
  if (n1 <= 0 || n2 <= 0) return GBDCT_ERR_INVALID_ARG;
  if (!pow2(n1) || !pow2(n2) || n1 < 2 || n2 < 2 || n1 > 16384 || n2 > 16384) return GBDCT_ERR_UNSUPPORTED;
  if (n1 * n2 > kNoAllocMaxElems) return GBDCT_ERR_UNSUPPORTED;

  float2* scratch = nullptr;
  const gbdct_status st = scratch_for_current_device(&scratch);
  if (st != GBDCT_OK) return st;

  const int N1 = (int)n1, N2 = (int)n2, l1 = lg2(n1), l2 = lg2(n2);
  const bool pair = l1 >= gbdct::kPairMinLog2 && l1 <= gbdct::kPairMaxLog2 && l2 >= gbdct::kPairMinLog2 &&
                    l2 <= gbdct::kPairMaxLog2;
  float2* work = scratch;
  float2* tw1 = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(scratch) + kWorkBytes);
  const int tot1 = gbdct::tw_size(N1), tot2 = gbdct::tw_size(N2);
  float2* tw2 = tw1 + up2(tot1 + 1);
  float2* fa = tw2 + up2(tot2 + 1);
  float2* fb = fa + up2(N1 / 2 + 1);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  if (tot1 > 0) k_na_stage_twiddles<<<(tot1 + 255) / 256, 256, 0, s>>>(tw1, N1, tot1);
  if (tot2 > 0) k_na_stage_twiddles<<<(tot2 + 255) / 256, 256, 0, s>>>(tw2, N2, tot2);
  const int nt = (N1 / 2 + 1 > N2) ? (N1 / 2 + 1) : N2;
  k_na_dct_tables<<<(nt + 255) / 256, 256, 0, s>>>(fa, fb, N1, N2);

  gbdct::Dct2dArgs a{};
  a.in = static_cast<const float*>(in);
  a.out = static_cast<float*>(out);
  a.work = work;
  a.n1 = N1;
  a.n2 = N2;
  a.in_bstride = a.out_bstride = (long long)N1 * N2;
  a.work_bstride = (long long)(N1 / 2) * N2;
  a.tw1 = tw1;
  a.tw2 = tw2;
  a.fa = fa;
  a.fb = fb;
  cudaError_t e;
  if (pair) {
    e = gbdct::run_fwd_cols2(l1, a, N2 / 4, 1, s, false);
    if (e == cudaSuccess) e = gbdct::run_fwd_rows2(l2, a, N1 / 4, 1, s, false);
  } else {
    gbdct::Dct2dArgs ac = a, ar = a;
    ac.seq_per_cta = gbdct::choose_seq_per_cta(N1, N2 / 2);
    ar.seq_per_cta = gbdct::choose_seq_per_cta(N2, N1 / 2);
    e = gbdct::run_fwd_cols(l1, ac, dim3((N2 / 2) / ac.seq_per_cta, 1), s, false);
    if (e == cudaSuccess) e = gbdct::run_fwd_rows(l2, ar, dim3((N1 / 2) / ar.seq_per_cta, 1), s, false);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? GBDCT_OK : GBDCT_ERR_CUDA;
}
