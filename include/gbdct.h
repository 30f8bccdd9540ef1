/*
 * gbdct.h - C ABI of the GB300 (sm_103a) multi-dimensional DCT library.
 *
 * The library computes the 2D DCT-II and its exact inverse by the three-stage
 * method of arXiv 2110.01172 (Section II-D, Algorithm 2; Section III): an
 * even/odd reorder of the real input (Eq. 2d_dct_pre), a 2D real-to-complex
 * FFT, and a twiddle-and-combine step that reads each conjugate-symmetric pair
 * once (Section III-B, Eqs. four-elements and s-t).  The inverse runs the
 * mirror image: the four-reads/two-writes twiddle preprocess (Eq. 2d_idct_pre),
 * a complex-to-real 2D FFT and the inverse reorder (Eq. 2d_idct_post).  The
 * reorder and the twiddle stages are fused into the first and last FFT passes,
 * so a 2D transform is two or three kernel launches (by kernel family; three
 * for the default four-step family) around one L2-resident intermediate.  The
 * same plans cover batches, 3D (Section III-D), the DST-II / IDXST kinds of
 * Section V-B, uneven-size batches, the spectral Poisson solve of Algorithm 4
 * and a split-BF16 tensor-core precision mode.
 *
 * Conventions (all arrays are dense, row-major, last axis contiguous):
 *   forward  X[k1,k2] = sum_{n1,n2} x[n1,n2] cos(pi k1 (2n1+1)/(2N1))
 *                                          cos(pi k2 (2n2+1)/(2N2))
 *            (unnormalised, Section II-A Eq. 2d-dct-definition);
 *   inverse  the exact inverse of the forward map, i.e. the paper's IDCT
 *            (DCT-III, Eq. 1b) applied per axis and scaled by 2/N per axis,
 *            so inverse(forward(x)) == x.
 *
 * Every function returns a gbdct_status; no C++ exception crosses the ABI.
 * Pointers named "device" must point to memory of the plan's CUDA device;
 * the exec calls also accept page-locked host buffers (see gbdct_exec_forward).
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * A plan may be used by one stream at a time (it owns one workspace).
 */
#ifndef GBDCT_H_
#define GBDCT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbdct_plan_s* gbdct_plan_t;

typedef enum gbdct_status {
  GBDCT_OK = 0,
  GBDCT_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, bad rank, dims <= 0 */
  GBDCT_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement */
  GBDCT_ERR_OOM = 3,          /* device allocation failed at plan creation */
  GBDCT_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
  GBDCT_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up */
} gbdct_status;

typedef enum gbdct_kind {
  /* forward: 2D DCT-II; inverse: its exact inverse (scaled DCT-III). */
  GBDCT_DCT2 = 0,
  /* forward: 2D DST-II X = sum x sin(pi(2n1+1)(k1+1)/2N1) sin(..N2); inverse:
     its exact inverse.  DST-II is not in the paper; it is computed through
     DST-II(x)_k = DCT-II((-1)^n x)_{N-1-k} on each axis. */
  GBDCT_DST2 = 1,
  /* inverse: IDCT on axis 0 and IDXST on axis 1 (Section V-B, Eq. idxst,
     "IDCT_IDXST"), with the same 2/N scaling as the DCT-II inverse.  IDXST
     ignores x_0, so the map is singular: exec_forward returns
     GBDCT_ERR_UNSUPPORTED for this kind. */
  GBDCT_IDCT_IDXST = 2,
  /* inverse: IDXST on axis 0 and IDCT on axis 1 ("IDXST_IDCT"); inverse only,
     like GBDCT_IDCT_IDXST. */
  GBDCT_IDXST_IDCT = 3
} gbdct_kind;

typedef enum gbdct_dtype {
  GBDCT_F32 = 0               /* float32 input and output, float32 arithmetic */
} gbdct_dtype;

typedef enum gbdct_precision {
  GBDCT_PREC_FP32 = 0,        /* default: the FFT kernels, FP32 arithmetic */
  GBDCT_PREC_SPLIT_BF16 = 1   /* dense DFT-GEMMs on the tensor cores, bf16 hi+lo split, FP32 accumulation */
} gbdct_precision;

/* Human-readable name of a status code (static storage, never NULL). */
const char* gbdct_status_string(gbdct_status status);

/* Library version string, e.g. "gbdct 0.1.0 sm_103a" (static storage). */
const char* gbdct_version(void);

/*
 * Create a plan for one transform of shape dims[0] x ... x dims[ndim-1] on the
 * current CUDA device (Algorithm 2 "Require": a real N1 x N2 matrix).  The
 * plan precomputes every twiddle table in FP64 on the device and rounds it to
 * FP32 (the paper's coefficients "fixed before the call", Section III-B), and
 * allocates its workspace (gbdct_plan_workspace_bytes).
 *   out   receives the plan handle (unchanged on error).
 *   ndim  2, or 3 for the 3D DCT-II and its inverse (kind GBDCT_DCT2 only;
 *         the triple separable sum, Section III-D).  A 3D plan of dims
 *         (N0, N1, N2) runs the 2D transform of each of its N0 slices as one
 *         batched 2D plan and a 1D pass along axis 0 (inverse: axis 0 first);
 *         N0 must be a power of two between 2 and 4096 and batch * N0 at most
 *         65535, else GBDCT_ERR_UNSUPPORTED.  ndim 1 gives UNSUPPORTED.
 *   dims  ndim sizes; each must be a power of two between 2 and 16384, else
 *         GBDCT_ERR_UNSUPPORTED (dims <= 0 give GBDCT_ERR_INVALID_ARG).
 *   kind  a gbdct_kind; dtype must be GBDCT_F32.  In the two-pass (tp) and
 *         four-step (fs2) families the index/sign maps of the other kinds are
 *         folded into the first loads and last stores of the DCT-II kernels; the other
 *         families run the DCT-II kernels between two index/sign map kernels
 *         and own an extra staging array of batch*N1*N2 floats.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.  Synchronises the device.
 */
gbdct_status gbdct_plan_create(gbdct_plan_t* out, int ndim, const int64_t* dims,
                               int kind, int dtype);

/*
 * As gbdct_plan_create, for `batch` independent transforms of the same shape
 * stored back to back (batch >= 1); one exec call processes all of them in the
 * same launches.  The workspace grows linearly with `batch`.
 */
gbdct_status gbdct_plan_create_batched(gbdct_plan_t* out, int ndim, const int64_t* dims,
                                       int64_t batch, int kind, int dtype);

/*
 * Forward transform.  `in` and `out` point to batch * prod(dims) float32
 * values, 16-byte aligned; in == out (in place) is allowed.  Each may be
 * memory of the plan's device, managed memory, or page-locked host memory
 * (cudaHostAlloc / cudaHostRegister, mapped at the same address): host
 * buffers are read and written by the transform's own first and last kernels
 * over the host link, with no staging copy (a two-pass plan runs such calls
 * with its four-step launches, which access whole row segments, where that
 * family supports the shape; results then differ from the device-buffer call
 * in FP32 rounding only).  Pageable host memory is accepted
 * only where the device can access it (cudaDevAttrPageableMemoryAccess).  The
 * call is asynchronous on `stream`; the caller keeps both buffers alive until
 * the stream has passed the work.  Errors: INVALID_ARG (NULL, misaligned or
 * inaccessible pointer — e.g. another device's memory — NULL plan), CUDA
 * (launch failure).
 */
gbdct_status gbdct_exec_forward(gbdct_plan_t plan, const void* in, void* out, void* stream);

/* Inverse transform; same contract as gbdct_exec_forward. */
gbdct_status gbdct_exec_inverse(gbdct_plan_t plan, const void* in, void* out, void* stream);

/*
 * Diagnostic: runs launch `step` (0 <= step < gbdct_plan_launches_per_exec) of
 * the forward (inverse = 0) or inverse (inverse = 1) sequence alone, reading
 * and writing the same buffers the full call would.  Used to time each kernel
 * of a transform on its own stream; the result of a single step is an
 * intermediate, not a transform.  Errors: INVALID_ARG (NULL plan, step out of
 * range, NULL/misaligned pointers), UNSUPPORTED, CUDA.
 */
gbdct_status gbdct_exec_step(gbdct_plan_t plan, int inverse, int step, const void* in, void* out, void* stream);

/* Short description of launch `step` (static storage; "" when out of range). */
const char* gbdct_plan_step_name(gbdct_plan_t plan, int inverse, int step);

/* Bytes of device workspace owned by the plan: the intermediate array, the
 * staging array of mapped kinds (see gbdct_plan_create) and the DFT-GEMM
 * operands of the split-BF16 mode (0 for a NULL plan).  Twiddle tables are not
 * counted. */
size_t gbdct_plan_workspace_bytes(gbdct_plan_t plan);

/* Number of kernel launches one exec call issues (0 for a NULL plan). */
int gbdct_plan_launches_per_exec(gbdct_plan_t plan);

/* Name of the kernel family the plan runs ("seq", "pair", "fs2" or "tp"; ""
 * for a NULL plan).  Every family computes the same transform; the plan picks
 * the fastest one that supports the shape (tp: both sides in 128..8192, two
 * launches per direction, the default for N1 <= 4096; fs2: N1 in 256..8192
 * and N2 in 256..16384, three launches; pair: both sides in 16..8192; seq:
 * any supported size), and the environment variable
 * GBDCT_KERNEL_FAMILY=seq|pair|fs2|tp, read at plan creation, forces a family
 * when it supports the shape (for testing and comparison). */
const char* gbdct_plan_kernel_family(gbdct_plan_t plan);

/* Reports (and clears) a failure recorded on the device by the plan's
 * kernels: the pipelined tensor-core kernels of the split-BF16 mode bound every
 * wait on an asynchronous copy or MMA, and a wait that gives up records it
 * here instead of hanging the GPU (the kernel then waits for the work it has
 * already issued and leaves its output tile unwritten, so the transform's
 * output is invalid).  Synchronises with the device.  Returns GBDCT_OK,
 * GBDCT_ERR_TIMEOUT, GBDCT_ERR_INVALID_ARG (NULL plan) or GBDCT_ERR_CUDA. */
gbdct_status gbdct_plan_check_device_error(gbdct_plan_t plan);

/* Magnitude threshold of Section V-A (Eq. image-compression, the compression
 * step of Algorithm 3), fused into the forward transform's last stores: every
 * forward output X with |X| < eps (compared in FP32) is stored as zero.
 * eps = 0 (the default) turns it off; the inverse is unaffected.  Supported for
 * 2D plans of the two-pass ("tp") and four-step ("fs2") families with
 * N2 <= 8192, else
 * GBDCT_ERR_UNSUPPORTED; INVALID_ARG for a NULL plan or a negative or NaN eps. */
gbdct_status gbdct_plan_set_threshold(gbdct_plan_t plan, float eps);

/* Bound of every device-side wait of the plan's pipelined kernels, in polls of
 * the waited-on barrier (0, the default, is about half a second; a 3D plan
 * passes it to its 2D slices).  A diagnostic: a tiny bound makes the waits
 * give up, which is how the timeout path (gbdct_plan_check_device_error) is
 * tested without a device fault.  Errors: INVALID_ARG (NULL plan). */
gbdct_status gbdct_plan_set_wait_limit(gbdct_plan_t plan, uint32_t polls);

/* Release the plan and its device memory.  NULL is accepted (no-op).  The
 * caller must make sure no stream still uses the plan. */
gbdct_status gbdct_plan_destroy(gbdct_plan_t plan);

/*
 * As gbdct_plan_create_batched with the kernel family named by `family`
 * ("seq", "pair", "fs2", "tp", or "fs2/<A>" for the four-step family with
 * the column split N1 = A * (N1 / A), A and N1 / A in {16, 32, 64, 128}; every
 * family computes the same transform).  Errors: INVALID_ARG (NULL or unknown name, and the checks of
 * gbdct_plan_create_batched), UNSUPPORTED when that family does not support
 * the shape, OOM, CUDA.  For a 3D plan the family applies to its 2D slices.
 */
gbdct_status gbdct_plan_create_family(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                      int dtype, const char* family);

/*
 * Autotuned plan: times one forward + inverse (inverse only for the
 * inverse-only kinds) of every candidate that supports the shape and batch —
 * the kernel families and their tile parameters ("fs2/<A>" four-step splits,
 * "tp/<NP>" two-pass strip widths) — on scratch buffers it allocates and frees, with CUDA events on a private
 * stream, and returns the plan of the fastest.  The choice is cached for the
 * process and, when the environment variable GBDCT_TUNE_CACHE names a file,
 * appended to that file ("key family microseconds" lines) and read back by
 * later processes, which then create the plan without timing.  family_out
 * (optional, family_cap bytes) receives the chosen candidate's name.
 * Synchronises the device.  Errors as gbdct_plan_create_batched.
 */
gbdct_status gbdct_plan_create_tuned(gbdct_plan_t* out, int ndim, const int64_t* dims, int64_t batch, int kind,
                                     int dtype, char* family_out, size_t family_cap);

/*
 * Precision mode of a plan.  GBDCT_PREC_SPLIT_BF16 evaluates the separable
 * definition as dense products, X = C1 x C2^T forward and x = D1 X D2^T
 * inverse (C the DCT-II matrix, D its exact inverse), on the tensor cores by
 * a hand-written tcgen05 kernel: every operand is split into bf16 hi + lo
 * parts and each product is accumulated in FP32 (in tensor memory) as
 * hi*hi + hi*lo + lo*hi.  Its error is that of the split (about 5e-6 relative
 * in L2, stated per result), not the FP32 path's.  Supported for 2D GBDCT_DCT2
 * plans with both sides between 128 and 2048 (UNSUPPORTED otherwise); the
 * first switch allocates the matrices (FP64-generated, split once) and four
 * bf16 arrays of batch*N1*N2 and synchronises the device.  gbdct_exec_step is
 * UNSUPPORTED in this mode.  GBDCT_PREC_FP32 switches back.
 * Errors: INVALID_ARG (NULL plan, unknown mode), UNSUPPORTED, OOM, CUDA.
 */
gbdct_status gbdct_plan_set_precision(gbdct_plan_t plan, int precision);

/*
 * Uneven-size batches of 2D transforms (the batch parallelism of Section IV:
 * independent transforms are independent units of work).  The executor groups
 * the `count` transforms by shape into batched plans and defines a packed
 * layout: transform i starts gbdct_multi_offset(m, i) floats into a buffer of
 * gbdct_multi_total_elems(m) floats (groups back to back, largest shapes
 * first; every offset is a multiple of 4 floats).  One exec transforms every
 * transform of the packed input into the same place of the packed output.
 *   shapes  count (N1, N2) pairs, each side a power of two in [2, 16384].
 *   kind    a gbdct_kind (the inverse-only kinds reject forward execs).
 *   flags   GBDCT_MULTI_GRAPH: the first exec for a given (in, out,
 *           direction) captures the whole fork/join of the groups as one CUDA
 *           graph, later execs with the same pointers replay it (one launch);
 *           up to 8 graphs are kept.  Capture needs the calling thread to have
 *           no other capture in progress.
 *           GBDCT_MULTI_TUNE: each group's plan comes from
 *           gbdct_plan_create_tuned (plan creation takes longer).
 * Exec is asynchronous on `stream`: the groups run on the executor's own
 * streams between a fork and a join on `stream`.  An executor may be used by
 * one stream at a time.  Errors: INVALID_ARG (NULL, count < 1, dims <= 0,
 * unknown kind or flags, misaligned pointers), UNSUPPORTED (a shape outside the
 * limits; forward of an inverse-only kind), OOM, CUDA.
 */
typedef struct gbdct_multi_s* gbdct_multi_t;
#define GBDCT_MULTI_GRAPH 1
#define GBDCT_MULTI_TUNE 2
gbdct_status gbdct_multi_create(gbdct_multi_t* out, int count, const int64_t* shapes, int kind, int flags);
/* The packed layout gbdct_multi_create would use, computed on the host with
 * no CUDA call: offsets[i] (optional, count entries) receives the offset in
 * floats of transform i, *groups (optional) the number of shape groups.
 * Returns the floats in a packed buffer, or -1 for invalid shapes. */
int64_t gbdct_multi_layout(int count, const int64_t* shapes, int64_t* offsets, int* groups);
/* Offset (floats) of transform `index` in the packed buffers; -1 if out of range or NULL. */
int64_t gbdct_multi_offset(gbdct_multi_t m, int index);
/* Floats in a packed buffer (0 for NULL). */
int64_t gbdct_multi_total_elems(gbdct_multi_t m);
/* Number of shape groups (batched plans); 0 for NULL. */
int gbdct_multi_group_count(gbdct_multi_t m);
/* Kernel family of group `group`'s plan ("" if out of range). */
const char* gbdct_multi_group_family(gbdct_multi_t m, int group);
/* Forward (inverse = 0) or inverse transform of every transform in the packed buffers. */
gbdct_status gbdct_multi_exec(gbdct_multi_t m, int inverse, const void* in, void* out, void* stream);
/* Releases the executor, its plans, streams and graphs (NULL accepted). */
gbdct_status gbdct_multi_destroy(gbdct_multi_t m);

/*
 * Spectral Neumann Poisson solve of Section V-B, Algorithm 4 (the electrostatic
 * step of analytical placement).  For a density map rho (N1 x N2 float32):
 *   a    = DCT-II(rho)                                   (forward, as above)
 *   psi  = IDCT2(a / (wu^2 + wv^2))                      potential
 *   xi0  = IDXST_IDCT(a wu / (wu^2 + wv^2))              field along axis 0
 *   xi1  = IDCT_IDXST(a wv / (wu^2 + wv^2))              field along axis 1
 * with wu = pi u / N1, wv = pi v / N2 and the (0,0) term set to zero (the paper
 * only says "scaled a1, a2"; these are the eigenfrequencies of the cosine
 * basis in grid units).  The solver owns three plans (DCT2, IDXST_IDCT,
 * IDCT_IDXST), the wu / wv tables and an N1 x N2 table of the eigenvalue
 * denominators 1 / (wu^2 + wv^2), all evaluated in FP64 at creation and
 * rounded once to FP32.  Calls switch to the solver's device for their
 * duration.
 */
typedef struct gbdct_poisson_s* gbdct_poisson_t;

/* Shape limits as gbdct_plan_create (powers of two, 2..16384). */
gbdct_status gbdct_poisson_create(gbdct_poisson_t* out, int64_t n1, int64_t n2);

/* rho, psi, xi0, xi1: device float32 arrays of N1*N2, 16-byte aligned; psi, xi0
 * and xi1 must be distinct (rho may alias psi).  Asynchronous on `stream`; a
 * solver may be used by one stream at a time. */
gbdct_status gbdct_poisson_solve(gbdct_poisson_t p, const void* rho, void* psi, void* xi0, void* xi1,
                                 void* stream);

/* Device bytes owned by the solver (workspaces, staging and tables). */
size_t gbdct_poisson_workspace_bytes(gbdct_poisson_t p);

/* Releases the solver (NULL accepted). */
gbdct_status gbdct_poisson_destroy(gbdct_poisson_t p);

/*
 * Forward 2D DCT-II (same result as gbdct_exec_forward with a GBDCT_DCT2 plan)
 * that allocates no device memory.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate on the call path - code
 * running inside a host framework that owns all device memory through its own
 * pool and forbids raw cudaMalloc, or latency-critical loops where a
 * cudaMalloc/cudaFree (which may synchronise the whole device) would stall
 * other streams.  Instead of a plan, the workspace and the twiddle tables live
 * in one static device array of 5 MiB that every GPU which loads the library
 * holds until the process exits; each call rebuilds the tables in it and then
 * runs the two fused passes.
 *   in, out  device pointers to n1*n2 float32 values, 16-byte aligned
 *            (in == out allowed).
 *   n1, n2   powers of two in [2, 16384] with n1*n2 <= 2^20 (1 Mi elements,
 *            e.g. 1024 x 1024); larger sizes return GBDCT_ERR_UNSUPPORTED,
 *            dims <= 0 return GBDCT_ERR_INVALID_ARG.
 *   stream   cudaStream_t as void* (NULL = legacy default stream).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and sets kernel
 * attributes; make that first call before any stream capture.  Calls issue no
 * cudaMalloc, cudaFree or allocating library routine.  All calls on a device
 * share the one array, which keeps the last call's contents: calls whose
 * kernels overlap on the GPU (different streams, no ordering between them)
 * race and give wrong results, so order them on one stream or with events.
 */
gbdct_status gbdct_dct2d_forward_noalloc(const void* in, void* out, int64_t n1, int64_t n2, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBDCT_H_ */
