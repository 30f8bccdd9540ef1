// dct_axis0.cuh - 1D DCT-II and its exact inverse along the outermost axis of
// a row-major (N, M) float32 array (M contiguous), for the 3D transform.
//
// The 3D DCT-II is separable (Section III-D): the library runs the 2D
// transform of every (N1, N2) slice, then this pass along axis 0 over the
// M = N1 * N2 columns (inverse: this pass first, then the 2D inverses).  Along
// the axis it is the 1D three-stage method (Section III-A, Eqs. n_pre/n_post)
// on two real columns at once:
//   forward  z[n] = x[s(n), 2p] + i x[s(n), 2p+1],   s(n) = 2n (n <= (N-1)/2),
//                                                      2N - 2n - 1 otherwise
//            Z = FFT_N(z);  Va[k] = (Z[k] + conj Z[N-k]) / 2,
//                           Vb[k] = (Z[k] - conj Z[N-k]) / (2i)
//            X_a[k] = Re(e^{-i pi k / 2N} Va[k]),  X_b likewise
//   inverse  Va[k] = e^{+i pi k / 2N} (X_a[k] - i X_a[N-k]) / N   (X_a[N] = 0)
//            z = IFFT_N(Va + i Vb);  x[s(n), 2p] = Re z[n], x[s(n), 2p+1] = Im z[n]
// One CTA holds all N rows of a strip of columns in shared memory and writes
// the same strip back (so the pass may run in place).  For N >= 64 (the
// packed form) a float4 of a row, two adjacent column pairs, is one two-lane
// sequence of the packed-FP32x2 Stockham engine (fft_soa.cuh), NP such
// sequences per CTA interleaved point by point so that a warp's loads and
// stores cover 32/NP rows x NP*16 contiguous bytes; below 64 one CTA holds P
// column pairs as one complex sequence each (fft_core.cuh, sequence stride
// odd so that a warp reading one row across sequences is conflict-free).
#pragma once

#include <cuda_runtime.h>

namespace gbdct {

struct AxisArgs {
  const float* in;
  float* out;
  long long M;          // real columns (contiguous extent)
  long long bstride;    // floats between batch items
  const float2* tw;     // stage twiddles of the length-N FFT (pmax 16)
  const float4* tw4;    // the same as (wr, wr, wi, wi), for the packed two-lane form
  const float2* w;      // forward: e^{-i pi k / 2N} / 2; inverse: e^{+i pi k / 2N} / N  (k < N)
  int lgP;              // log2 of the column pairs per CTA
};

constexpr int kAxisMinLog2 = 1, kAxisMaxLog2 = 12;

// Column pairs per CTA for a length-N axis over M real columns: up to 32, with
// the tile (P sequences of ~1.125 N complex) kept near 74 KB.
inline int axis0_lgP(int lgN, long long M) {
  int lg = 13 - lgN;  // P * N <= 8192
  if (lg > 5) lg = 5;
  if (lg < 0) lg = 0;
  while (lg > 0 && (2LL << lg) > M) --lg;
  return lg;
}

size_t axis0_smem_bytes(int lgN, int lgP);
int axis0_threads(int lgN, int lgP);

// prepare=true raises the dynamic shared-memory limit of both directions' kernels.
cudaError_t run_axis0(int lgN, bool inverse, const AxisArgs& a, int batch, cudaStream_t s, bool prepare);

}  // namespace gbdct
