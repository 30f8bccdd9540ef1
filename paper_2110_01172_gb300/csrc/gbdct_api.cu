// gbdct_api.cu - plans, FP64 twiddle generation and the C ABI (include/gbdct.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/gbdct.h"
#include "dct2d_launch.cuh"
#include "dct_axis0.cuh"
#include "gemm_path.cuh"

using gbdct::Dct2dArgs;

struct gbdct_plan_s {
  int ndim;
  int64_t dims[3];
  int64_t batch;
  int kind;
  int device;
  int n1, n2, lg1, lg2;
  float2* tables;   // one allocation holding every twiddle table
  size_t table_elems;
  float2* work;     // half-spectrum workspace, batch * (N1/2) * N2 complex
  size_t work_bytes;
  Dct2dArgs args;   // pointers and sizes shared by all passes
  int b_cols, b_rows;  // sequences per CTA of the column and row passes
  int family;          // kernel family (FAM_*)
  float2* fstw;        // four-step twiddles W_N1^{n1a k1b} (FAM_FS2)
  int* err;            // device error word (bounded waits that gave up)
  bool host_fs2;       // two-pass plan that runs full transforms on host-mapped buffers with the four-step kernels
  int nsm;             // multiprocessors of the plan's device
  float* tmp;          // variant kinds: staging array (batch * N1 * N2 floats)
  int pmax;            // points per thread of the stage structure (twiddle layout)
  // ndim == 3 (N0, N1, N2): the 2D transforms of the N0 slices run as a batched
  // 2D plan, then a 1D pass along axis 0 (inverse: axis 0 first).
  gbdct_plan_t inner;  // batched 2D plan of the (N1, N2) slices (batch * N0 transforms)
  float2* ax_tables;   // axis-0 stage twiddles, forward post and inverse pre tables
  const float2* ax_fw; // e^{-i pi k / 2 N0} / 2
  const float2* ax_iw; // e^{+i pi k / 2 N0} / N0
  gbdct::AxisArgs ax;  // axis-0 pass arguments (in, out, w set per call)
  int lg0;
  int precision;             // GBDCT_PREC_FP32 (FFT kernels) or GBDCT_PREC_SPLIT_BF16
  gbdct::GemmPath* gemm;     // split-BF16 DFT-GEMM state (precision mode only)
  uint32_t wait_polls;       // bound of device-side waits (0: default), see gbdct_plan_set_wait_limit
};

namespace {

// Kernel families (all compute the same transform; chosen by size):
//   FAM_TP   two passes per direction: half-length column FFTs on strips +
//            row passes with the radix-2 column step folded in,
//            N1 in {512..8192}, N2 in {256..8192}
//   FAM_FS2  four-step column steps + two-item row passes (three passes),
//            N1 in {256..8192}, N2 in {256..16384}
//   FAM_PAIR two interleaved sequences per thread, 16 <= N1, N2 <= 8192
//   FAM_SEQ  one sequence per thread group, any supported size
enum { FAM_SEQ = 0, FAM_PAIR = 1, FAM_FS2 = 5, FAM_TP = 6 };

// Families whose kernels fold the other kinds' index/sign maps into their
// loads and stores (no map kernels, no staging array).
bool folds_maps(int family) { return family == FAM_FS2 || family == FAM_TP; }

// Radix-2 twiddles of the two-pass family: out[k] = W_N1^k, k in [0, N1/2], FP64.
__global__ void k_gen_r2_twiddles(float2* out, int n1) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n1 / 2) return;
  double sn, cs;
  sincospi(-2.0 * (double)k / (double)n1, &sn, &cs);
  out[k] = make_float2((float)cs, (float)sn);
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// The stage twiddles of length L again as (wr, wr, wi, wi), for the two-lane
// (packed FP32x2) FFT engine of fft_soa.cuh.
__global__ void k_expand_twiddles(const float2* __restrict__ tw, float4* out, int total) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const float2 w = tw[idx];
  out[idx] = make_float4(w.x, w.x, w.y, w.y);
}

// Stage twiddles of the Stockham FFT of length L (layout in fft_core.cuh):
// entry (j-1)*NS + k of the stage starting at NS is exp(-2 pi i j k / (NS R)),
// evaluated in FP64 from the exactly reduced integer j k mod (NS R).
__global__ void k_gen_stage_twiddles(float2* out, int L, int pmax, int total) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int off = 0;
  for (int ns = 1; ns < L; ns *= gbdct::stage_radix_p(L, ns, pmax)) {
    const int R = gbdct::stage_radix_p(L, ns, pmax);
    if (ns == 1) continue;
    const int sz = (R - 1) * ns;
    if (idx < off + sz) {
      const int e = idx - off;
      const long long j = e / ns + 1, k = e % ns;
      const long long M = (long long)ns * R;
      const long long m = (j * k) % M;
      double sn, cs;
      sincospi(-2.0 * (double)m / (double)M, &sn, &cs);
      out[idx] = make_float2((float)cs, (float)sn);
      return;
    }
    off += sz;
  }
}

// DCT twiddles (Section III-B, Eq. s-t: a = e^{-i pi n1/2N1}, b = e^{-i pi n2/2N2}):
//   fa[k] = a_k,                      k in [0, N1/2]
//   fb[k] = b_k / 2,                  k in [0, N2)      (the 1/2 of the combine)
//   ia[k] = conj(a_k) / (N1 N2),      k in [0, N1/2]    (inverse DFT scale folded in)
//   ib[k] = conj(b_k),                k in [0, N2)
__global__ void k_gen_dct_tables(float2* fa, float2* fb, float2* ia, float2* ib, int n1, int n2) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx <= n1 / 2) {
    double sn, cs;
    sincospi((double)idx / (2.0 * (double)n1), &sn, &cs);
    fa[idx] = make_float2((float)cs, (float)(-sn));
    const double sc = 1.0 / ((double)n1 * (double)n2);
    ia[idx] = make_float2((float)(cs * sc), (float)(sn * sc));
  }
  if (idx < n2) {
    double sn, cs;
    sincospi((double)idx / (2.0 * (double)n2), &sn, &cs);
    fb[idx] = make_float2((float)(0.5 * cs), (float)(-0.5 * sn));
    ib[idx] = make_float2((float)cs, (float)sn);
  }
}

// Axis-0 tables of the 3D transform (FP64, k in [0, N)):
//   fw[k] = e^{-i pi k / 2N} / 2   (forward post, Hermitian-split 1/2 folded in)
//   iw[k] = e^{+i pi k / 2N} / N   (inverse pre, inverse DFT scale folded in)
__global__ void k_gen_axis_tables(float2* fw, float2* iw, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double sn, cs;
  sincospi((double)k / (2.0 * (double)n), &sn, &cs);
  fw[k] = make_float2((float)(0.5 * cs), (float)(-0.5 * sn));
  iw[k] = make_float2((float)(cs / n), (float)(sn / n));
}

// Four-step twiddles W_N1^{n1a k1b} at n1a * B + k1b (n1a < A, k1b < B), FP64.
__global__ void k_gen_fs_twiddles(float2* out, int n1, int A, int B) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A * B) return;
  const long long m = ((long long)(idx / B) * (idx % B)) % n1;
  double sn, cs;
  sincospi(-2.0 * (double)m / (double)n1, &sn, &cs);
  out[idx] = make_float2((float)cs, (float)sn);
}

// Index map used by the DST-II and IDXST kinds around the DCT-II core:
// out(i, j) = sign(i, j) * in(src(i), src(j)) where, per axis, src(i) is i,
// N-1-i (reversal) or N-i with src(0) -> 0 value (the IDXST shift x_{N-n},
// x_N = 0, Section V-B Eq. idxst), and sign is (-1)^i on the flagged axes.
struct MapSpec {
  int rev0, rev1, shift0, shift1, sgn0, sgn1;
};

__global__ void k_map2d(const float* __restrict__ in, float* __restrict__ out, int n1, int n2, long long bs,
                        MapSpec m) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= n2) return;
  const float* src = in + (long long)blockIdx.z * bs;
  float* dst = out + (long long)blockIdx.z * bs;
  const int si = m.rev0 ? n1 - 1 - i : (m.shift0 ? (i ? n1 - i : -1) : i);
  const int sj = m.rev1 ? n2 - 1 - j : (m.shift1 ? (j ? n2 - j : -1) : j);
  float v = (si < 0 || sj < 0) ? 0.f : src[(long long)si * n2 + sj];
  if (((m.sgn0 & i) ^ (m.sgn1 & j)) & 1) v = -v;
  dst[(long long)i * n2 + j] = v;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

gbdct_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GBDCT_OK;
  if (e == cudaErrorMemoryAllocation) return GBDCT_ERR_OOM;
  return GBDCT_ERR_CUDA;
}

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      switched = (cudaSetDevice(dev) == cudaSuccess);
    }
  }
  ~DeviceGuard() {
    if (switched) cudaSetDevice(prev);
  }
};

// True when kernels on `device` may dereference `ptr`: this device's memory,
// managed memory, page-locked host memory mapped at the same address (read
// and written over the host link by the kernels themselves), or any host
// memory when the device can access pageable memory.  While `s` is capturing
// a graph the check is skipped (the pointers of a captured launch are the
// caller's own device buffers, and the query is not needed there).
// Returns 0 (not accessible), 1 (this device's memory) or 2 (accessible
// otherwise); *is_dev tells the kernels whether bulk tensor copies may be used.
enum { PTR_NONE = 0, PTR_DEVICE = 1, PTR_OTHER = 2 };
int pointer_kind(const void* ptr, int device, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone) return PTR_DEVICE;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return PTR_NONE;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == device ? PTR_DEVICE : PTR_NONE;
    case cudaMemoryTypeManaged: return PTR_OTHER;
    case cudaMemoryTypeHost: return at.devicePointer == ptr ? PTR_OTHER : PTR_NONE;
    default: {
      int pageable = 0;
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
      return pageable != 0 ? PTR_OTHER : PTR_NONE;
    }
  }
}

void free_plan(gbdct_plan_s* p) {
  if (!p) return;
  if (p->inner) gbdct_plan_destroy(p->inner);
  if (p->gemm) gbdct::gemm_destroy(p->gemm);
  if (p->ax_tables) cudaFree(p->ax_tables);
  if (p->tables) cudaFree(p->tables);
  if (p->work) cudaFree(p->work);
  if (p->tmp) cudaFree(p->tmp);
  delete p;
}

}  // namespace

extern "C" {
static gbdct_status exec2d(gbdct_plan_t p, const void* in, void* out, void* stream, bool inverse, int step);
}

static gbdct_status run_plan(gbdct_plan_t p, bool inverse, int step, const void* in, void* out,
                                           cudaStream_t s) {
  return exec2d(p, in, out, reinterpret_cast<void*>(s), inverse, step);
}

static gbdct_status create_impl(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                int dtype, const char* force);

static gbdct_status create_3d(gbdct_plan_t* out, const int64_t* dims, int64_t batch, int kind, int dtype,
                              const char* force) {
  if (kind != GBDCT_DCT2) return GBDCT_ERR_UNSUPPORTED;
  for (int i = 0; i < 3; ++i)
    if (!is_pow2(dims[i])) return GBDCT_ERR_UNSUPPORTED;
  const int lg0 = ilog2(dims[0]);
  if (lg0 < gbdct::kAxisMinLog2 || lg0 > gbdct::kAxisMaxLog2) return GBDCT_ERR_UNSUPPORTED;
  if (batch * dims[0] > 65535) return GBDCT_ERR_UNSUPPORTED;
  gbdct_plan_s* p = new (std::nothrow) gbdct_plan_s();
  if (!p) return GBDCT_ERR_OOM;
  p->ndim = 3;
  for (int i = 0; i < 3; ++i) p->dims[i] = dims[i];
  p->batch = batch;
  p->kind = kind;
  p->lg0 = lg0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return GBDCT_ERR_CUDA;
  }
  gbdct_status st = create_impl(&p->inner, 2, dims + 1, batch * dims[0], GBDCT_DCT2, dtype, force);
  if (st != GBDCT_OK) {
    free_plan(p);
    return st;
  }
  const int n0 = (int)dims[0];
  const int tot = gbdct::tw_size_p(n0, 16);
  const size_t t0 = round_up(tot + 1, 2), tn = round_up(n0, 2);
  // stage twiddles (float2, then the same as float4 for the packed form), forward post, inverse pre
  cudaError_t e = cudaMalloc(&p->ax_tables, (3 * t0 + 2 * tn) * sizeof(float2));
  float4* tw4 = nullptr;
  if (e == cudaSuccess) {
    float2* fw = p->ax_tables + t0;
    float2* iw = fw + tn;
    tw4 = reinterpret_cast<float4*>(iw + tn);
    if (tot > 0) {
      k_gen_stage_twiddles<<<(tot + 255) / 256, 256>>>(p->ax_tables, n0, 16, tot);
      k_expand_twiddles<<<(tot + 255) / 256, 256>>>(p->ax_tables, tw4, tot);
    }
    k_gen_axis_tables<<<(n0 + 255) / 256, 256>>>(fw, iw, n0);
    p->ax_fw = fw;
    p->ax_iw = iw;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  p->ax.M = dims[1] * dims[2];
  p->ax.bstride = dims[0] * dims[1] * dims[2];
  p->ax.tw = p->ax_tables;
  p->ax.tw4 = tw4;
  p->ax.lgP = gbdct::axis0_lgP(lg0, p->ax.M);
  if (e == cudaSuccess) e = gbdct::run_axis0(lg0, false, p->ax, 1, 0, true);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }
  p->work_bytes = gbdct_plan_workspace_bytes(p->inner);
  p->family = p->inner->family;
  *out = p;
  return GBDCT_OK;
}

static gbdct_status exec3d(gbdct_plan_t p, const void* in, void* out, cudaStream_t s, bool inverse, int step) {
  const int ni = gbdct_plan_launches_per_exec(p->inner);
  gbdct::AxisArgs ax = p->ax;
  ax.w = inverse ? p->ax_iw : p->ax_fw;
  if (!inverse) {
    if (step < 0 || step < ni) {
      const gbdct_status st = run_plan(p->inner, false, step, in, out, s);
      if (st != GBDCT_OK) return st;
    }
    if (step >= 0 && step != ni) return GBDCT_OK;
    ax.in = static_cast<const float*>(out);
    ax.out = static_cast<float*>(out);
    return cuda_status(gbdct::run_axis0(p->lg0, false, ax, (int)p->batch, s, false));
  }
  if (step < 0 || step == 0) {
    ax.in = static_cast<const float*>(in);
    ax.out = static_cast<float*>(out);
    const cudaError_t e = gbdct::run_axis0(p->lg0, true, ax, (int)p->batch, s, false);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (step == 0) return GBDCT_OK;
  return run_plan(p->inner, true, step < 0 ? -1 : step - 1, out, out, s);
}

extern "C" {

const char* gbdct_status_string(gbdct_status status) {
  switch (status) {
    case GBDCT_OK: return "GBDCT_OK";
    case GBDCT_ERR_INVALID_ARG: return "GBDCT_ERR_INVALID_ARG";
    case GBDCT_ERR_UNSUPPORTED: return "GBDCT_ERR_UNSUPPORTED";
    case GBDCT_ERR_OOM: return "GBDCT_ERR_OOM";
    case GBDCT_ERR_CUDA: return "GBDCT_ERR_CUDA";
    case GBDCT_ERR_TIMEOUT: return "GBDCT_ERR_TIMEOUT";
  }
  return "GBDCT_ERR_UNKNOWN";
}

const char* gbdct_version(void) { return "gbdct 0.1.0 sm_103a"; }

gbdct_status gbdct_plan_create_batched(gbdct_plan_t* out, int ndim, const int64_t* dims,
                                       int64_t batch, int kind, int dtype) {
  return create_impl(out, ndim, dims, batch, kind, dtype, nullptr);
}

gbdct_status gbdct_plan_create_family(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                      int dtype, const char* family) {
  if (!family) return GBDCT_ERR_INVALID_ARG;
  return create_impl(out, ndim, dims, batch, kind, dtype, family);
}

}  // extern "C"

// force: a family name that must be used (UNSUPPORTED if it does not support
// the shape), or NULL for the default choice (GBDCT_KERNEL_FAMILY may override
// it when the named family supports the shape).
static gbdct_status create_impl(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                int dtype, const char* force) {
  if (!out || !dims || batch < 1) return GBDCT_ERR_INVALID_ARG;
  if (ndim < 1 || ndim > 3) return GBDCT_ERR_INVALID_ARG;
  for (int i = 0; i < ndim; ++i)
    if (dims[i] <= 0) return GBDCT_ERR_INVALID_ARG;
  if (kind < GBDCT_DCT2 || kind > GBDCT_IDXST_IDCT) return GBDCT_ERR_INVALID_ARG;
  if (dtype != GBDCT_F32) return GBDCT_ERR_UNSUPPORTED;
  // a family name, "fs2/<A>" for the four-step family with the split
  // N1 = A * (N1 / A) of its column FFT (A and N1 / A in {16, 32, 64, 128}),
  // or "tp/<NP>" for the two-pass family with column strips of NP column pairs
  const char* fname = force ? force : getenv("GBDCT_KERNEL_FAMILY");
  int split_a = 0, strip_np = 0;
  if (fname && strncmp(fname, "fs2/", 4) == 0) {
    split_a = atoi(fname + 4);
    if (split_a != 16 && split_a != 32 && split_a != 64 && split_a != 128) split_a = -1;
  }
  if (fname && strncmp(fname, "tp/", 3) == 0) {
    strip_np = atoi(fname + 3);
    if (strip_np < 1 || strip_np > 32 || (strip_np & (strip_np - 1))) strip_np = -1;
  }
  if (force && (split_a < 0 || strip_np < 0 ||
                (!split_a && !strip_np && strcmp(force, "seq") && strcmp(force, "pair") && strcmp(force, "fs2") &&
                 strcmp(force, "tp"))))
    return GBDCT_ERR_INVALID_ARG;
  if (split_a < 0) split_a = 0;
  if (strip_np < 0) strip_np = 0;
  if (ndim == 3) return create_3d(out, dims, batch, kind, dtype, force);
  if (ndim != 2) return GBDCT_ERR_UNSUPPORTED;
  for (int i = 0; i < ndim; ++i) {
    if (!is_pow2(dims[i])) return GBDCT_ERR_UNSUPPORTED;
    const int lg = ilog2(dims[i]);
    if (lg < gbdct::kMinLog2 || lg > gbdct::kMaxLog2) return GBDCT_ERR_UNSUPPORTED;
  }
  if (batch > 65535) return GBDCT_ERR_UNSUPPORTED;

  gbdct_plan_s* p = new (std::nothrow) gbdct_plan_s();
  if (!p) return GBDCT_ERR_OOM;
  p->ndim = ndim;
  for (int i = 0; i < 3; ++i) p->dims[i] = i < ndim ? dims[i] : 1;
  p->batch = batch;
  p->kind = kind;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return GBDCT_ERR_CUDA;
  }
  const int n1 = (int)dims[0], n2 = (int)dims[1];
  p->n1 = n1;
  p->n2 = n2;
  p->lg1 = ilog2(n1);
  p->lg2 = ilog2(n2);

  const bool pair = p->lg1 >= gbdct::kPairMinLog2 && p->lg1 <= gbdct::kPairMaxLog2 &&
                    p->lg2 >= gbdct::kPairMinLog2 && p->lg2 <= gbdct::kPairMaxLog2;
  const bool fs2 = p->lg1 >= gbdct::kFs2MinLog2N1 && p->lg1 <= gbdct::kFs2MaxLog2N1 &&
                   p->lg2 >= gbdct::kFs2MinLog2N2 && p->lg2 <= gbdct::kFs2MaxLog2N2;
  const bool tp = p->lg1 >= gbdct::kTpMinLog2N1 && p->lg1 <= gbdct::kTpMaxLog2N1 &&
                  p->lg2 >= gbdct::kTpMinLog2N2 && p->lg2 <= gbdct::kTpMaxLog2N2;
  // a strip width the two-pass column pass is built for at this shape
  const bool tp_np_ok = tp && strip_np > 0 && gbdct::tp_strip_ok(n1 / 2, n2, strip_np);
  // Default: the two-pass family for N1 <= 4096, the four-step family where
  // it applies, else the two-sequence family, else one sequence per thread
  // group (fastest measured at every shape they share: e.g. 128^2 11.9 vs
  // 15.8 us (pair), 256^2 11.8 vs 16.5 (fs2), 4096^2 69.5 vs 76.3; at
  // N1 = 8192 the four-step column steps beat the two-pass column pass, whose
  // strips there are 32 bytes of 4096 rows, where they apply: 8192 x 128 runs
  // two-pass, 18 / 20 us vs 27 / 30 us with pair).
  p->family = (tp && (p->lg1 <= 12 || !fs2)) ? FAM_TP : fs2 ? FAM_FS2 : (pair ? FAM_PAIR : FAM_SEQ);
  // GBDCT_KERNEL_FAMILY=seq|pair|fs2 forces a family when it supports the shape
  // (used to test and compare every kernel family on the same inputs).
  if (const char* f = fname) {
    const int before = p->family;
    int chosen = -1;
    if (!strcmp(f, "seq")) chosen = FAM_SEQ;
    else if (!strcmp(f, "pair") && pair) chosen = FAM_PAIR;
    else if (!strcmp(f, "fs2") && fs2) chosen = FAM_FS2;
    else if (!strcmp(f, "tp") && tp) chosen = FAM_TP;
    else if (strip_np && tp_np_ok) chosen = FAM_TP;
    else if (split_a && fs2 && n1 / split_a >= 16 && n1 / split_a <= 128) chosen = FAM_FS2;
    if (chosen < 0 && force) {
      delete p;
      return GBDCT_ERR_UNSUPPORTED;
    }
    p->family = chosen < 0 ? before : chosen;
  }
  const bool two_pass = p->family == FAM_TP;
  // a two-pass plan also carries the four-step configuration: full transforms
  // on host-mapped buffers run the four-step kernels, whose first and last
  // launches read and write whole 1 KB row segments (the two-pass column
  // pass's 32-byte row pieces cross the host link poorly), where the
  // four-step family supports the shape
  p->host_fs2 = two_pass && fs2;
  const bool four_step = p->family == FAM_FS2 || p->host_fs2;
  const bool two_item_rows = four_step || two_pass;  // row passes on the SoA engine (float4 twiddles)
  p->pmax = 16;

  // Table layout, each block padded to 2 float2 (16 B).
  const int tot1 = gbdct::tw_size_p(n1, p->pmax), tot2 = gbdct::tw_size_p(n2, p->pmax);
  const size_t t1 = round_up(tot1 + 1, 2);
  const size_t t2 = round_up(tot2 + 1, 2);
  const size_t ta = round_up(n1 / 2 + 1, 2);
  const size_t tb = round_up(n2, 2);
  const size_t tf = four_step ? round_up(n1, 2) : 0;
  const size_t tx = two_item_rows ? 2 * t2 : 0;  // float4 copy of the N2 stage twiddles
  // two-pass family: stage twiddles of length N1/2 (float2 and float4 copies)
  // and the radix-2 twiddles W_N1^k
  const int totm = two_pass ? gbdct::tw_size_p(n1 / 2, p->pmax) : 0;
  const size_t tm = two_pass ? round_up(totm + 1, 2) : 0;
  const size_t tr = two_pass ? round_up(n1 / 2 + 1, 2) : 0;
  p->table_elems = t1 + t2 + 2 * ta + 2 * tb + tf + tx + 3 * tm + tr + 2;  // + 16 bytes for the error word
  cudaError_t e = cudaMalloc(&p->tables, p->table_elems * sizeof(float2));
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }
  float2* tw1 = p->tables;
  float2* tw2 = tw1 + t1;
  float2* fa = tw2 + t2;
  float2* ia = fa + ta;
  float2* fb = ia + ta;
  float2* ib = fb + tb;
  p->fstw = four_step ? ib + tb : nullptr;
  float4* tw2x = two_item_rows ? reinterpret_cast<float4*>(ib + tb + tf) : nullptr;
  float2* twm = two_pass ? ib + tb + tf + tx : nullptr;
  float4* tw1x = two_pass ? reinterpret_cast<float4*>(ib + tb + tf + tx + tm) : nullptr;
  float2* r2w = two_pass ? ib + tb + tf + tx + 3 * tm : nullptr;
  p->err = reinterpret_cast<int*>(ib + tb + tf + tx + 3 * tm + tr);

  p->work_bytes = (size_t)batch * (size_t)(n1 / 2) * (size_t)n2 * sizeof(float2);
  e = cudaMalloc(&p->work, p->work_bytes);
  // staging array for the map kernels of the other kinds (fs2 folds the maps in)
  if (e == cudaSuccess && kind != GBDCT_DCT2 && !folds_maps(p->family))
    e = cudaMalloc(&p->tmp, (size_t)batch * (size_t)n1 * (size_t)n2 * sizeof(float));
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }

  if (tot1 > 0) k_gen_stage_twiddles<<<(tot1 + 255) / 256, 256>>>(tw1, n1, p->pmax, tot1);
  if (tot2 > 0) k_gen_stage_twiddles<<<(tot2 + 255) / 256, 256>>>(tw2, n2, p->pmax, tot2);
  const int nt = (n1 / 2 + 1 > n2) ? (n1 / 2 + 1) : n2;
  k_gen_dct_tables<<<(nt + 255) / 256, 256>>>(fa, fb, ia, ib, n1, n2);
  int fsA = 0, fsB = 0;
  if (four_step) {
    gbdct::fs2_split(p->lg1, &fsA, &fsB);
    if (split_a && n1 / split_a >= 16 && n1 / split_a <= 128) {
      fsA = split_a;
      fsB = n1 / split_a;
    }
  }
  if (p->fstw) k_gen_fs_twiddles<<<(n1 + 255) / 256, 256>>>(p->fstw, n1, fsA, fsB);
  if (tw2x && tot2 > 0) k_expand_twiddles<<<(tot2 + 255) / 256, 256>>>(tw2, tw2x, tot2);
  if (two_pass) {
    if (totm > 0) {
      k_gen_stage_twiddles<<<(totm + 255) / 256, 256>>>(twm, n1 / 2, p->pmax, totm);
      k_expand_twiddles<<<(totm + 255) / 256, 256>>>(twm, tw1x, totm);
    }
    k_gen_r2_twiddles<<<(n1 / 2 + 256) / 256, 256>>>(r2w, n1);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemset(p->err, 0, 16);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }

  Dct2dArgs& a = p->args;
  a.n1 = n1;
  a.n2 = n2;
  a.in_bstride = (long long)n1 * n2;
  a.out_bstride = (long long)n1 * n2;
  a.work_bstride = (long long)(n1 / 2) * n2;
  a.work = p->work;
  a.tw1 = tw1;
  a.tw2 = tw2;
  a.tw2x = tw2x;
  a.tw1x = tw1x;
  a.r2w = r2w;
  a.fa = fa;
  a.fb = fb;
  a.ia = ia;
  a.ib = ib;
  a.fstw = p->fstw;
  a.err = p->err;
  a.step_filter = -1;
  a.fsA = fsA;
  a.fsB = fsB;
  a.tpNP = (two_pass && tp_np_ok) ? strip_np : 0;  // strip width of the column pass (0: default)
  a.vkind = folds_maps(p->family) ? kind : 0;
  a.nsm = p->nsm;
  p->b_cols = gbdct::choose_seq_per_cta(n1, n2 / 2);
  p->b_rows = gbdct::choose_seq_per_cta(n2, n1 / 2);

  // Raise the dynamic shared-memory limit of the kernels once.
  if (p->family == FAM_FS2) {
    e = gbdct::run_fs2(p->lg1, p->lg2, false, a, 1, 0, true);
  } else if (p->family == FAM_TP) {
    e = gbdct::run_tp(p->lg1, p->lg2, false, a, 1, 0, true);
    if (e == cudaSuccess && p->host_fs2) e = gbdct::run_fs2(p->lg1, p->lg2, false, a, 1, 0, true);
  } else if (p->family == FAM_PAIR) {
    e = gbdct::run_fwd_cols2(p->lg1, a, 1, 1, 0, true);
    if (e == cudaSuccess) e = gbdct::run_inv_cols2(p->lg1, a, 1, 1, 0, true);
    if (e == cudaSuccess) e = gbdct::run_fwd_rows2(p->lg2, a, 1, 1, 0, true);
    if (e == cudaSuccess) e = gbdct::run_inv_rows2(p->lg2, a, 1, 1, 0, true);
  } else {
    Dct2dArgs ac = a, ar = a;
    ac.seq_per_cta = p->b_cols;
    ar.seq_per_cta = p->b_rows;
    dim3 g(1, 1);
    e = gbdct::run_fwd_cols(p->lg1, ac, g, 0, true);
    if (e == cudaSuccess) e = gbdct::run_inv_cols(p->lg1, ac, g, 0, true);
    if (e == cudaSuccess) e = gbdct::run_fwd_rows(p->lg2, ar, g, 0, true);
    if (e == cudaSuccess) e = gbdct::run_inv_rows(p->lg2, ar, g, 0, true);
  }
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }
  *out = p;
  return GBDCT_OK;
}

extern "C" {

gbdct_status gbdct_plan_create(gbdct_plan_t* out, int ndim, const int64_t* dims, int kind,
                               int dtype) {
  return gbdct_plan_create_batched(out, ndim, dims, 1, kind, dtype);
}

static gbdct_status exec_core(gbdct_plan_t p, const void* in, void* out, cudaStream_t s, bool inverse,
                              int step = -1, bool io_dev = false);
static int core_launches(gbdct_plan_t p) {
  return p->family == FAM_FS2 ? 3 : 2;
}

static cudaError_t run_map(gbdct_plan_t p, const float* in, float* out, MapSpec m, cudaStream_t s) {
  const dim3 grid((p->n2 + 255) / 256, p->n1, (unsigned)p->batch);
  k_map2d<<<grid, 256, 0, s>>>(in, out, p->n1, p->n2, (long long)p->n1 * p->n2, m);
  return cudaGetLastError();
}

// DST-II and the IDXST kinds as index/sign maps around the DCT-II core:
//   DST-II(x)_k = DCT-II((-1)^n x)_{N-1-k} per axis (both axes);
//   IDXST(x)_k = (-1)^k IDCT({x_{N-n}})_k, x_N = 0 (Section V-B, Eq. idxst).
static gbdct_status exec2d(gbdct_plan_t p, const void* in, void* out, void* stream, bool inverse,
                           int step) {
  if (!p || !in || !out) return GBDCT_ERR_INVALID_ARG;
  if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u)) return GBDCT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int kin = pointer_kind(in, p->device, s), kout = pointer_kind(out, p->device, s);
  if (kin == PTR_NONE || kout == PTR_NONE) return GBDCT_ERR_INVALID_ARG;
  const bool io_dev = kin == PTR_DEVICE && kout == PTR_DEVICE;
  if (p->ndim == 3) return exec3d(p, in, out, s, inverse, step);
  if (p->precision == GBDCT_PREC_SPLIT_BF16)
    return step >= 0 ? GBDCT_ERR_UNSUPPORTED
                     : gbdct::gemm_exec(p->gemm, inverse, static_cast<const float*>(in), static_cast<float*>(out), s);
  if (p->kind == GBDCT_DCT2) return exec_core(p, in, out, s, inverse, step, io_dev);
  if (!inverse && (p->kind == GBDCT_IDCT_IDXST || p->kind == GBDCT_IDXST_IDCT)) return GBDCT_ERR_UNSUPPORTED;
  if (folds_maps(p->family)) return exec_core(p, in, out, s, inverse, step, io_dev);  // maps folded in (vkind)
  MapSpec pre{}, post{};
  if (p->kind == GBDCT_DST2) {
    if (!inverse) {
      pre.sgn0 = pre.sgn1 = 1;
      post.rev0 = post.rev1 = 1;
    } else {
      pre.rev0 = pre.rev1 = 1;
      post.sgn0 = post.sgn1 = 1;
    }
  } else {
    // IDXST ignores x_0, so the IDCT_IDXST / IDXST_IDCT maps are singular and
    // have no forward (inverse-of-inverse) transform.
    if (!inverse) return GBDCT_ERR_UNSUPPORTED;
    if (p->kind == GBDCT_IDCT_IDXST) {
      pre.shift1 = 1;
      post.sgn1 = 1;
    } else {
      pre.shift0 = 1;
      post.sgn0 = 1;
    }
  }
  const int nc = core_launches(p);
  if (step < 0 || step == 0) {
    const cudaError_t e = run_map(p, static_cast<const float*>(in), p->tmp, pre, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (step < 0 || (step >= 1 && step <= nc)) {
    const gbdct_status st = exec_core(p, p->tmp, p->tmp, s, inverse, step < 0 ? -1 : step - 1);
    if (st != GBDCT_OK) return st;
  }
  if (step < 0 || step == nc + 1) return cuda_status(run_map(p, p->tmp, static_cast<float*>(out), post, s));
  return GBDCT_OK;
}

static gbdct_status exec_core(gbdct_plan_t p, const void* in, void* out, cudaStream_t s, bool inverse,
                              int step, bool io_dev) {
  Dct2dArgs a = p->args;
  a.in = static_cast<const float*>(in);
  a.out = static_cast<float*>(out);
  a.step_filter = step;
  a.io_dev = io_dev ? 1 : 0;
  a.polls = p->wait_polls;
  const int batch = (int)p->batch;
  const bool s0 = step < 0 || step == 0, s1 = step < 0 || step == 1;
  cudaError_t e = cudaSuccess;
  if (p->family == FAM_FS2) {
    return cuda_status(gbdct::run_fs2(p->lg1, p->lg2, inverse, a, batch, s, false));
  }
  if (p->family == FAM_TP) {
    // host-mapped or managed buffers: the four-step kernels (full transforms
    // only; single steps keep the two-pass launch sequence)
    if (!io_dev && step < 0 && p->host_fs2)
      return cuda_status(gbdct::run_fs2(p->lg1, p->lg2, inverse, a, batch, s, false));
    return cuda_status(gbdct::run_tp(p->lg1, p->lg2, inverse, a, batch, s, false));
  }
  if (p->family == FAM_PAIR) {
    if (!inverse) {
      if (s0) e = gbdct::run_fwd_cols2(p->lg1, a, p->n2 / 4, batch, s, false);
      if (e == cudaSuccess && s1) e = gbdct::run_fwd_rows2(p->lg2, a, p->n1 / 4, batch, s, false);
    } else {
      if (s0) e = gbdct::run_inv_rows2(p->lg2, a, p->n1 / 4, batch, s, false);
      if (e == cudaSuccess && s1) e = gbdct::run_inv_cols2(p->lg1, a, p->n2 / 4, batch, s, false);
    }
    return cuda_status(e);
  }
  Dct2dArgs ac = a, ar = a;
  ac.seq_per_cta = p->b_cols;
  ar.seq_per_cta = p->b_rows;
  const dim3 gc((p->n2 / 2) / p->b_cols, batch);
  const dim3 gr((p->n1 / 2) / p->b_rows, batch);
  if (!inverse) {
    if (s0) e = gbdct::run_fwd_cols(p->lg1, ac, gc, s, false);
    if (e == cudaSuccess && s1) e = gbdct::run_fwd_rows(p->lg2, ar, gr, s, false);
  } else {
    if (s0) e = gbdct::run_inv_rows(p->lg2, ar, gr, s, false);
    if (e == cudaSuccess && s1) e = gbdct::run_inv_cols(p->lg1, ac, gc, s, false);
  }
  return cuda_status(e);
}

gbdct_status gbdct_exec_forward(gbdct_plan_t plan, const void* in, void* out, void* stream) {
  return exec2d(plan, in, out, stream, false, -1);
}

gbdct_status gbdct_exec_inverse(gbdct_plan_t plan, const void* in, void* out, void* stream) {
  return exec2d(plan, in, out, stream, true, -1);
}

gbdct_status gbdct_exec_step(gbdct_plan_t plan, int inverse, int step, const void* in, void* out, void* stream) {
  if (!plan || step < 0 || step >= gbdct_plan_launches_per_exec(plan)) return GBDCT_ERR_INVALID_ARG;
  return exec2d(plan, in, out, stream, inverse != 0, step);
}

const char* gbdct_plan_step_name(gbdct_plan_t plan, int inverse, int step) {
  if (!plan || step < 0 || step >= gbdct_plan_launches_per_exec(plan)) return "";
  if (plan->ndim == 3) {
    const int ni = gbdct_plan_launches_per_exec(plan->inner);
    if (!inverse) return step < ni ? gbdct_plan_step_name(plan->inner, 0, step)
                                   : "axis-0 pass (reorder + column FFT + split + twiddle)";
    return step == 0 ? "axis-0 pass (twiddle + column IFFT + inverse reorder)"
                     : gbdct_plan_step_name(plan->inner, 1, step - 1);
  }
  static const char* kFwd2[] = {"column pass (reorder + column FFT + split)",
                                "row pass (row FFT + symmetric-pair postprocess)"};
  static const char* kInv2[] = {"row pass (four-read preprocess + row IFFT)",
                                "column pass (column IFFT + inverse reorder)"};
  static const char* kFwdTp[] = {"column pass (reorder + half-length column FFTs)",
                                 "row pass (radix-2 step + split + row FFT + postprocess)"};
  static const char* kInvTp[] = {"row pass (preprocess + row IFFT + pairing + radix-2 step)",
                                 "column pass (half-length column IFFTs + inverse reorder)"};
  static const char* kFwd3[] = {"column step C1 (reorder + DFT_B + twiddle)", "column step C2 (DFT_A)",
                                "row pass (split + row FFT + postprocess)"};
  static const char* kInv3[] = {"row pass (preprocess + row IFFT + pairing)", "column step C2' (DFT_A + twiddle)",
                                "column step C1' (DFT_B + inverse reorder)"};
  const bool three = core_launches(plan) == 3;
  int k = step;
  if (plan->kind != GBDCT_DCT2 && !folds_maps(plan->family)) {
    if (k == 0) return "index/sign map (pre)";
    if (k == gbdct_plan_launches_per_exec(plan) - 1) return "index/sign map (post)";
    k -= 1;
  }
  if (three) return inverse ? kInv3[k] : kFwd3[k];
  if (plan->family == FAM_TP) return inverse ? kInvTp[k] : kFwdTp[k];
  return inverse ? kInv2[k] : kFwd2[k];
}

size_t gbdct_plan_workspace_bytes(gbdct_plan_t plan) {
  if (!plan) return 0;
  const size_t staging = plan->tmp ? (size_t)plan->batch * plan->n1 * plan->n2 * sizeof(float) : 0;
  return plan->work_bytes + staging + gbdct::gemm_workspace_bytes(plan->gemm);
}

gbdct_status gbdct_plan_set_precision(gbdct_plan_t plan, int precision) {
  if (!plan) return GBDCT_ERR_INVALID_ARG;
  if (precision == GBDCT_PREC_FP32) {
    plan->precision = GBDCT_PREC_FP32;  // the DFT-GEMM state is kept for a later switch back
    return GBDCT_OK;
  }
  if (precision != GBDCT_PREC_SPLIT_BF16) return GBDCT_ERR_INVALID_ARG;
  if (plan->ndim != 2 || plan->kind != GBDCT_DCT2) return GBDCT_ERR_UNSUPPORTED;
  if (plan->n1 > gbdct::kGemmMaxSide || plan->n2 > gbdct::kGemmMaxSide || plan->n1 < gbdct::kGemmMinSide ||
      plan->n2 < gbdct::kGemmMinSide || plan->batch > 65535)
    return GBDCT_ERR_UNSUPPORTED;
  if (!plan->gemm) {
    DeviceGuard guard(plan->device);
    gbdct_status st = GBDCT_OK;
    plan->gemm = gbdct::gemm_create(plan->n1, plan->n2, (int)plan->batch, plan->err, &st);
    if (!plan->gemm) return st;
    gbdct::gemm_set_wait_polls(plan->gemm, plan->wait_polls);
  }
  plan->precision = GBDCT_PREC_SPLIT_BF16;
  return GBDCT_OK;
}

int gbdct_plan_launches_per_exec(gbdct_plan_t plan) {
  if (!plan) return 0;
  if (plan->precision == GBDCT_PREC_SPLIT_BF16) return 3;  // split kernel + two tensor-core products
  if (plan->ndim == 3) return gbdct_plan_launches_per_exec(plan->inner) + 1;
  const int core = core_launches(plan);
  return (plan->kind == GBDCT_DCT2 || folds_maps(plan->family)) ? core : core + 2;
}

const char* gbdct_plan_kernel_family(gbdct_plan_t plan) {
  if (!plan) return "";
  switch (plan->family) {
    case FAM_TP: return "tp";
    case FAM_FS2: return "fs2";
    case FAM_PAIR: return "pair";
  }
  return "seq";
}

gbdct_status gbdct_plan_set_threshold(gbdct_plan_t plan, float eps) {
  if (!plan || !(eps >= 0.f)) return GBDCT_ERR_INVALID_ARG;
  if (plan->ndim != 2 || !folds_maps(plan->family) || plan->n2 > 8192) return GBDCT_ERR_UNSUPPORTED;
  plan->args.thresh = eps;
  return GBDCT_OK;
}

gbdct_status gbdct_plan_set_wait_limit(gbdct_plan_t plan, uint32_t polls) {
  if (!plan) return GBDCT_ERR_INVALID_ARG;
  if (plan->ndim == 3) return gbdct_plan_set_wait_limit(plan->inner, polls);
  plan->wait_polls = polls;
  gbdct::gemm_set_wait_polls(plan->gemm, polls);
  return GBDCT_OK;
}

gbdct_status gbdct_plan_check_device_error(gbdct_plan_t plan) {
  if (!plan) return GBDCT_ERR_INVALID_ARG;
  if (plan->ndim == 3) return gbdct_plan_check_device_error(plan->inner);
  DeviceGuard guard(plan->device);
  int v = 0;
  if (cudaMemcpy(&v, plan->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GBDCT_ERR_CUDA;
  if (v == 0) return GBDCT_OK;
  const int zero = 0;
  cudaMemcpy(plan->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
  return GBDCT_ERR_TIMEOUT;
}

gbdct_status gbdct_plan_destroy(gbdct_plan_t plan) {
  if (!plan) return GBDCT_OK;
  DeviceGuard guard(plan->device);
  free_plan(plan);
  return GBDCT_OK;
}

}  // extern "C"
