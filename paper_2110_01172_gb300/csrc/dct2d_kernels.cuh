// dct2d_kernels.cuh - the two fused passes of the 2D DCT-II and of its inverse.
//
// Method: arXiv 2110.01172, Section II-D / Algorithm 2 and Section III.  With
// v = x reordered by Eq. (2d_dct_pre) and V = DFT2(v),
//   X[k1,k2] = 1/2 Re( b_k2 (a_k1 V(k1,k2) + conj(a_k1) V(N1-k1 mod N1, k2)) )
// where a_k = e^{-i pi k / 2N1}, b_k = e^{-i pi k / 2N2} (Eq. 2d_dct_post with
// the factor 1/2 and the periodic index that make it equal Eq. 2d-dct-
// definition).  The four outputs (k1,k2), (N1-k1,k2), (k1,N2-k2),
// (N1-k1,N2-k2) come from the same two spectrum values (Eqs. four-elements,
// s-t): with s = b(aP + conj(a)Q), t = b(aP - conj(a)Q) they are Re s/2,
// -Im t/2, -Im s/2 and -Re t/2.
//
// Data flow (forward), columns first so that the output is written as whole
// rows:
//   pass C  (fwd_cols)  per CTA: B "complex columns" p, each the pair of input
//           columns (2p, 2p+1).  Column 2p of x is column p of v and column
//           2p+1 is column N2-1-p of v (Eq. 2d_dct_pre), so the pair is one
//           complex sequence z = v(:,p) + i v(:,N2-1-p), loaded with the row
//           reorder of Eq. (2d_dct_pre) applied to the row index.  One complex
//           FFT of length N1 gives both real-column spectra, which are split
//           by Hermitian symmetry and stored in the half-spectrum workspace
//           Wk[k1][n2] (k1 < N1/2), row 0 packing the two real rows k1 = 0 and
//           k1 = N1/2 as re/im.
//   pass R  (fwd_rows)  per CTA: B workspace rows k1.  A complex FFT of
//           length N2 gives V(k1, :) for all k2, and V(N1-k1, k2) =
//           conj V(k1, N2-k2) (Hermitian symmetry of the 2D real DFT,
//           Section II-D), so the twiddle/combine postprocess of rows k1 and
//           N1-k1 needs only this row: it is fused into the epilogue and both
//           output rows are written whole.
// The inverse runs the mirror image: pass R' reads input rows k1 and N1-k1,
// applies the four-read twiddle preprocess (Eq. 2d_idct_pre, with the
// conjugated twiddle and the 1/(N1 N2) of the inverse DFT folded into the
// a-table), runs the inverse row FFT and writes the workspace; pass C' rebuilds
// the full Hermitian column from the half spectrum, runs the inverse column
// FFT of two real columns at once and stores them with the inverse reorder of
// Eq. (2d_idct_post).
#pragma once

#include "fft_core.cuh"

namespace gbdct {

struct Dct2dArgs {
  const float* in;
  float* out;
  float2* work;
  int n1, n2;
  long long in_bstride, out_bstride, work_bstride;  // per-transform strides (elements)
  const float2* tw1;  // stage twiddles for length N1
  const float2* tw2;  // stage twiddles for length N2
  const float2* fa;   // a_k1, k1 in [0, N1/2]
  const float2* fb;   // b_k2 / 2, k2 in [0, N2)
  const float2* ia;   // conj(a_k1) / (N1 N2), k1 in [0, N1/2]
  const float2* ib;   // conj(b_k2), k2 in [0, N2)
  int seq_per_cta;    // B
  const float2* fstw; // four-step twiddles W_N1^{n1a k1b} (four-step family only)
  int* err;           // device error word: set to 1 by a bounded wait that gave up
  int step_filter;    // host side only: -1 runs every launch, k runs launch k alone
  int fsA, fsB;       // four-step split N1 = A * B (four-step families)
  int vkind;          // kind whose index/sign maps the fs2 kernels fold into their
                      // loads and stores (0: DCT-II, no map; see dct2d_fs2_kernels.cuh)
  const float4* tw2x; // stage twiddles for length N2 as (wr, wr, wi, wi) (two-item row passes)
  float thresh;       // forward outputs with |X| < thresh stored as zero (0: off; two-item row passes)
  const float4* tw1x; // stage twiddles for length N1/2 as (wr, wr, wi, wi) (two-pass column passes)
  const float2* r2w;  // W_N1^k = exp(-2 pi i k / N1), k in [0, N1/2] (two-pass family's radix-2 step)
  int tpNP;           // strip width of the two-pass column pass in column pairs (0: the default)
  uint32_t polls;     // bound of device-side waits in polls (0: the default)
  int io_dev;         // host side only: input and output are device memory (bulk tensor copies allowed)
  int nsm;            // host side only: multiprocessors of the device
};

template <int L>
__host__ __device__ constexpr int max_threads_for() { return L >= 16384 ? 1024 : 512; }

// Row of the input that lands at position n of the reordered sequence
// (Eq. 2d_dct_pre): 2n for n <= (L-1)/2, else 2L - 2n - 1.
__device__ __forceinline__ int reorder_src(int n, int L) { return (n <= ((L - 1) >> 1)) ? 2 * n : 2 * L - 2 * n - 1; }
// Inverse map: position of input row r in the reordered sequence.
__device__ __forceinline__ int reorder_dst(int r, int L) { return (r & 1) ? (L - 1 - (r >> 1)) : (r >> 1); }

// ----------------------------------------------------------------------------
// Forward pass C: reorder + column FFT + real-pair split -> workspace
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(max_threads_for<L>())
k_fwd_cols(Dct2dArgs a) {
  extern __shared__ float4 smem_f4[];
  float2* sm = reinterpret_cast<float2*>(smem_f4);
  constexpr int TPS = fft_tps(L);
  constexpr int LP = pad_len<float2>(L);
  const int B = a.seq_per_cta;
  const int N2 = a.n2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int p0 = blockIdx.x * B;
  const float* x = a.in + (long long)blockIdx.y * a.in_bstride;
  float2* W = a.work + (long long)blockIdx.y * a.work_bstride;

  for (int i = tid; i < L * B; i += nthr) {
    const int b = i % B, r = i / B;
    const float2 z = __ldg(reinterpret_cast<const float2*>(x + (long long)r * N2 + 2 * (p0 + b)));
    sm[b * LP + pidx<float2>(reorder_dst(r, L))] = z;
  }
  __syncthreads();
  cta_fft<L, false>(sm + (tid / TPS) * LP, tid % TPS, a.tw1);

  // Z = FFT(u + i w) with u = v(:,p), w = v(:,N2-1-p) real:
  //   U[k] = (Z[k] + conj Z[L-k]) / 2,  Wt[k] = (Z[k] - conj Z[L-k]) / (2i).
  for (int i = tid; i < (L / 2) * B; i += nthr) {
    const int b = i % B, k = i / B;
    const float2* s = sm + b * LP;
    const int p = p0 + b;
    float2 u, w;
    if (k == 0) {
      const float2 z0 = s[pidx<float2>(0)];
      const float2 zh = s[pidx<float2>(L / 2)];
      u = make_float2(z0.x, zh.x);  // U[0], U[L/2] are real: packed re/im
      w = make_float2(z0.y, zh.y);
    } else {
      const float2 zk = s[pidx<float2>(k)];
      const float2 zm = s[pidx<float2>(L - k)];
      u = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      w = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
    W[(long long)k * N2 + p] = u;
    W[(long long)k * N2 + (N2 - 1 - p)] = w;
  }
}

// ----------------------------------------------------------------------------
// Forward pass R: row FFT + twiddle/symmetric-pair postprocess -> output rows
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(max_threads_for<L>())
k_fwd_rows(Dct2dArgs a) {
  extern __shared__ float4 smem_f4[];
  float2* sm = reinterpret_cast<float2*>(smem_f4);
  constexpr int TPS = fft_tps(L);
  constexpr int LP = pad_len<float2>(L);
  const int B = a.seq_per_cta;
  const int N1 = a.n1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int r0 = blockIdx.x * B;
  const float2* W = a.work + (long long)blockIdx.y * a.work_bstride;
  float* y = a.out + (long long)blockIdx.y * a.out_bstride;

  for (int i = tid; i < L * B; i += nthr) {
    const int b = i / L, c = i % L;
    sm[b * LP + pidx<float2>(c)] = W[(long long)(r0 + b) * L + c];
  }
  __syncthreads();
  cta_fft<L, false>(sm + (tid / TPS) * LP, tid % TPS, a.tw2);

  constexpr int H = L / 2 + 1;  // k2 in [0, L/2]
  for (int i = tid; i < H * B; i += nthr) {
    const int b = i / H, k2 = i % H;
    const int k1 = r0 + b;
    const float2* s = sm + b * LP;
    const float2 Y = s[pidx<float2>(k2)];
    const float2 Ym = s[pidx<float2>((L - k2) & (L - 1))];
    const float2 bt = __ldg(a.fb + k2);  // b_k2 / 2
    const bool mirror = (k2 != 0) && (k2 != L / 2);
    if (k1 == 0) {
      // packed row: V(0,k2) = (Y + conj Ym)/2, V(N1/2,k2) = (Y - conj Ym)/(2i)
      const float2 sum = make_float2(Y.x + Ym.x, Y.y - Ym.y);   // 2 V(0,k2)
      const float2 dif = make_float2(Y.y + Ym.y, Ym.x - Y.x);   // 2 V(N1/2,k2)
      const float2 s0 = cmul(bt, sum);                           // b/2 (aP + conj(a)Q), a=1, P=Q
      constexpr float RH = 0.70710678118654752f;                 // (a + conj a)/2, a = e^{-i pi/4}
      const float2 sh = cmul(bt, make_float2(RH * dif.x, RH * dif.y));
      float* row0 = y;
      float* rowh = y + (long long)(N1 / 2) * L;
      row0[k2] = s0.x;
      rowh[k2] = sh.x;
      if (mirror) {
        row0[L - k2] = -s0.y;
        rowh[L - k2] = -sh.y;
      }
    } else {
      const float2 P = Y;
      const float2 Q = conjf2(Ym);
      const float2 av = __ldg(a.fa + k1);
      const float2 aP = cmul(av, P);
      const float2 aQ = cmulc(Q, av);  // conj(a) Q
      const float2 sv = cmul(bt, cadd(aP, aQ));
      const float2 tv = cmul(bt, csub(aP, aQ));
      float* rowa = y + (long long)k1 * L;
      float* rowb = y + (long long)(N1 - k1) * L;
      rowa[k2] = sv.x;
      rowb[k2] = -tv.y;
      if (mirror) {
        rowa[L - k2] = -sv.y;
        rowb[L - k2] = -tv.x;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Inverse pass R': four-read twiddle preprocess + inverse row FFT -> workspace
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(max_threads_for<L>())
k_inv_rows(Dct2dArgs a) {
  extern __shared__ float4 smem_f4[];
  float2* sm = reinterpret_cast<float2*>(smem_f4);
  constexpr int TPS = fft_tps(L);
  constexpr int LP = pad_len<float2>(L);
  const int B = a.seq_per_cta;
  const int N1 = a.n1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int r0 = blockIdx.x * B;
  const float* C = a.in + (long long)blockIdx.y * a.in_bstride;
  float2* W = a.work + (long long)blockIdx.y * a.work_bstride;

  constexpr int H = L / 2 + 1;
  for (int i = tid; i < H * B; i += nthr) {
    const int b = i / H, k2 = i % H;
    const int k1 = r0 + b;
    float2* s = sm + b * LP;
    const bool mirror = (k2 != 0) && (k2 != L / 2);
    const int km = (L - k2) & (L - 1);
    const float2 bk = __ldg(a.ib + k2);
    const float2 bm = __ldg(a.ib + km);
    if (k1 == 0) {
      // rows 0 and h = N1/2 (C(N1, .) = 0 for row 0; row h pairs with itself)
      const int h = N1 / 2;
      const float* c0 = C;
      const float* ch = C + (long long)h * L;
      const float c01 = c0[k2], c02 = k2 ? c0[km] : 0.f;  // C(., N2) = 0
      const float ch1 = ch[k2], ch2 = k2 ? ch[km] : 0.f;
      const float2 a0 = __ldg(a.ia + 0);
      const float2 ah = __ldg(a.ia + h);
      // V(0,k2) = a0 b [c01 - i c02];  V(h,k2) = ah b [(ch1-ch2) - i(ch1+ch2)]
      const float2 v0 = cmul(a0, cmul(bk, make_float2(c01, -c02)));
      const float2 vh = cmul(ah, cmul(bk, make_float2(ch1 - ch2, -(ch1 + ch2))));
      s[pidx<float2>(k2)] = make_float2(v0.x - vh.y, v0.y + vh.x);  // V(0) + i V(h)
      if (mirror) {
        const float2 w0 = cmul(a0, cmul(bm, make_float2(c02, -c01)));
        const float2 wh = cmul(ah, cmul(bm, make_float2(ch2 - ch1, -(ch2 + ch1))));
        s[pidx<float2>(km)] = make_float2(w0.x - wh.y, w0.y + wh.x);
      }
    } else {
      const float* ca = C + (long long)k1 * L;
      const float* cb = C + (long long)(N1 - k1) * L;
      const float c1 = ca[k2];
      const float c4 = k2 ? ca[km] : 0.f;  // C(., N2) = 0
      const float c3 = cb[k2];
      const float c2 = k2 ? cb[km] : 0.f;
      const float2 av = __ldg(a.ia + k1);
      // V(k1,k2)    = a b [(c1 - c2) - i (c3 + c4)]
      // V(k1,N2-k2) = a b'[(c4 - c3) - i (c2 + c1)]
      s[pidx<float2>(k2)] = cmul(av, cmul(bk, make_float2(c1 - c2, -(c3 + c4))));
      if (mirror) s[pidx<float2>(km)] = cmul(av, cmul(bm, make_float2(c4 - c3, -(c2 + c1))));
    }
  }
  __syncthreads();
  cta_fft<L, true>(sm + (tid / TPS) * LP, tid % TPS, a.tw2);

  for (int i = tid; i < L * B; i += nthr) {
    const int b = i / L, c = i % L;
    W[(long long)(r0 + b) * L + c] = sm[b * LP + pidx<float2>(c)];
  }
}

// ----------------------------------------------------------------------------
// Inverse pass C': Hermitian rebuild + inverse column FFT + inverse reorder
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(max_threads_for<L>())
k_inv_cols(Dct2dArgs a) {
  extern __shared__ float4 smem_f4[];
  float2* sm = reinterpret_cast<float2*>(smem_f4);
  constexpr int TPS = fft_tps(L);
  constexpr int LP = pad_len<float2>(L);
  const int B = a.seq_per_cta;
  const int N2 = a.n2;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int p0 = blockIdx.x * B;
  const float2* W = a.work + (long long)blockIdx.y * a.work_bstride;
  float* x = a.out + (long long)blockIdx.y * a.out_bstride;

  for (int i = tid; i < (L / 2) * B; i += nthr) {
    const int b = i % B, k = i / B;
    const int p = p0 + b;
    float2* s = sm + b * LP;
    const float2 wp = W[(long long)k * N2 + p];
    const float2 wq = W[(long long)k * N2 + (N2 - 1 - p)];
    if (k == 0) {
      s[pidx<float2>(0)] = make_float2(wp.x, wq.x);
      s[pidx<float2>(L / 2)] = make_float2(wp.y, wq.y);
    } else {
      // Z(k) = U(k,p) + i U(k,q);  Z(L-k) = conj U(k,p) + i conj U(k,q)
      s[pidx<float2>(k)] = make_float2(wp.x - wq.y, wp.y + wq.x);
      s[pidx<float2>(L - k)] = make_float2(wp.x + wq.y, wq.x - wp.y);
    }
  }
  __syncthreads();
  cta_fft<L, true>(sm + (tid / TPS) * LP, tid % TPS, a.tw1);

  for (int i = tid; i < L * B; i += nthr) {
    const int b = i % B, n = i / B;
    const float2 z = sm[b * LP + pidx<float2>(n)];
    *reinterpret_cast<float2*>(x + (long long)reorder_src(n, L) * N2 + 2 * (p0 + b)) = z;
  }
}

}  // namespace gbdct
