// fft_core.cuh - CTA-level batched complex FFT in shared memory (sm_103a).
//
// The FFT stage of the three-stage method (arXiv 2110.01172, Algorithm 2,
// "2D_RFFT") is computed here by hand-written radix-16/8/4/2 Stockham stages
// instead of a vendor library.  A CTA holds `B` sequences of length L in
// shared memory; every thread keeps P = min(L, 16) points in registers during
// a stage, so one stage is: gather P points from shared memory, multiply by
// the stage twiddles, run radix-R DFTs in registers, scatter the results back
// in autosorted (natural) order.  L = 16^a * r, with the radix-r stage last.
//
// Stage twiddles are read from a per-length FP32 table that the plan builds in
// FP64: the stage that starts at sub-transform size NS (> 1) with radix R owns
// (R-1)*NS entries, entry (j-1)*NS + k = exp(-2 pi i j k / (NS R)), so a warp
// reads consecutive k (coalesced) for each j.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbdct {

// ----------------------------------------------------------------------------
// Compile-time geometry
// ----------------------------------------------------------------------------

__host__ __device__ constexpr int fft_points(int L) { return L >= 16 ? 16 : L; }
__host__ __device__ constexpr int fft_tps(int L) { return L / fft_points(L); }
// Shared-memory row length in float2: two float2 of padding after every 16.
__host__ __device__ constexpr int pad_len(int L) { return L >= 16 ? L + (L >> 3) : L; }
__host__ __device__ constexpr int stage_radix(int L, int ns) { return (L / ns >= 16) ? 16 : (L / ns); }

// Offset (in float2) of the twiddle block of the stage that starts at `ns`.
__host__ __device__ constexpr int tw_offset(int L, int ns) {
  int off = 0;
  for (int n = 1; n < ns; n *= stage_radix(L, n)) {
    if (n > 1) off += (stage_radix(L, n) - 1) * n;
  }
  return off;
}
__host__ __device__ constexpr int tw_size(int L) { return tw_offset(L, L); }

__device__ __forceinline__ int pidx(int i) { return i + ((i >> 4) << 1); }

// ----------------------------------------------------------------------------
// Complex helpers (float2 = re, im)
// ----------------------------------------------------------------------------

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Multiply by the unit root e^{-i pi/2} (forward) or e^{+i pi/2} (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_mj(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Multiply by W16^E = exp(-+ 2 pi i E / 16) for a compile-time E in [0, 16).
template <int E, bool INV>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
  constexpr float RH = 0.70710678118654752f;  // sqrt(1/2)
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return mul_mj<INV>(a);
  } else if constexpr (e == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (e == 12) {
    return mul_mj<!INV>(a);
  } else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
    // odd multiples of pi/4: (+-RH, +-RH)
    constexpr float cr = (e == 2 || e == 14) ? RH : -RH;
    constexpr float ci0 = (e == 2 || e == 6) ? -RH : RH;  // forward imaginary part
    constexpr float ci = INV ? -ci0 : ci0;
    return make_float2(cr * a.x - ci * a.y, cr * a.y + ci * a.x);
  } else {
    constexpr int q = e & 3;                   // 1 or 3 within the quadrant
    constexpr float c0 = (q == 1) ? C1 : S1;   // |cos| of the base angle e*pi/8 mod pi/2
    constexpr float s0 = (q == 1) ? S1 : C1;
    // angle = e * pi / 8: quadrant e/4 rotates (c0, s0) by multiples of pi/2.
    constexpr int quad = e >> 2;
    constexpr float cs = (quad == 0) ? c0 : (quad == 1) ? -s0 : (quad == 2) ? -c0 : s0;
    constexpr float sn = (quad == 0) ? s0 : (quad == 1) ? c0 : (quad == 2) ? -s0 : -c0;
    // forward twiddle = cos - i sin; inverse = cos + i sin
    constexpr float wi = INV ? sn : -sn;
    return make_float2(fmaf(cs, a.x, -wi * a.y), fmaf(cs, a.y, wi * a.x));
  }
}

// ----------------------------------------------------------------------------
// Radix-R DFTs in registers (X_m = sum_j a_j W_R^{jm}, W_R = e^{-+2 pi i/R})
// ----------------------------------------------------------------------------

template <bool INV>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  const float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const float2 t2 = cadd(a1, a3), t3 = mul_mj<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<1, false>(float2*) {}
template <>
__device__ __forceinline__ void dft<1, true>(float2*) {}

template <>
__device__ __forceinline__ void dft<2, false>(float2* v) { dft2<false>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<2, true>(float2* v) { dft2<true>(v[0], v[1]); }

template <>
__device__ __forceinline__ void dft<4, false>(float2* v) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* v) { dft4<true>(v[0], v[1], v[2], v[3]); }

// 8 = 2 x 4: DFT4 on even and odd points, twiddle W8^k, radix-2 combine.
template <bool INV>
__device__ __forceinline__ void dft8_impl(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = mul_w16<2, INV>(o1);
  o2 = mul_w16<4, INV>(o2);
  o3 = mul_w16<6, INV>(o3);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* v) { dft8_impl<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* v) { dft8_impl<true>(v); }

// 16 = 4 x 4: column DFT4s over n1 (stride 4), twiddles W16^{n2 k1}, row DFT4s.
template <bool INV>
__device__ __forceinline__ void dft16_impl(float2* v) {
  dft4<INV>(v[0], v[4], v[8], v[12]);
  dft4<INV>(v[1], v[5], v[9], v[13]);
  dft4<INV>(v[2], v[6], v[10], v[14]);
  dft4<INV>(v[3], v[7], v[11], v[15]);
  // after the first layer v[n2 + 4 k1] = F_{n2}[k1]
  v[5] = mul_w16<1, INV>(v[5]);
  v[9] = mul_w16<2, INV>(v[9]);
  v[13] = mul_w16<3, INV>(v[13]);
  v[6] = mul_w16<2, INV>(v[6]);
  v[10] = mul_w16<4, INV>(v[10]);
  v[14] = mul_w16<6, INV>(v[14]);
  v[7] = mul_w16<3, INV>(v[7]);
  v[11] = mul_w16<6, INV>(v[11]);
  v[15] = mul_w16<9, INV>(v[15]);
  // row DFT4 over n2 for each k1; output index k1 + 4 k2
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a0 = v[4 * k1 + 0], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
    dft4<INV>(a0, a1, a2, a3);
    t[k1 + 0] = a0;
    t[k1 + 4] = a1;
    t[k1 + 8] = a2;
    t[k1 + 12] = a3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}
template <>
__device__ __forceinline__ void dft<16, false>(float2* v) { dft16_impl<false>(v); }
template <>
__device__ __forceinline__ void dft<16, true>(float2* v) { dft16_impl<true>(v); }

// ----------------------------------------------------------------------------
// Stockham stages over one sequence in shared memory
// ----------------------------------------------------------------------------

// Runs the stages from sub-transform size NS to L on the sequence at `s`
// (padded layout, natural order in and out).  `g` in [0, fft_tps(L)) is the
// thread's rank within the sequence; every thread of the CTA must call this
// (it contains __syncthreads), each with its own sequence pointer.
template <int L, int NS, bool INV>
__device__ __forceinline__ void fft_stages(float2* __restrict__ s, int g,
                                           const float2* __restrict__ tw) {
  if constexpr (NS < L) {
    constexpr int R = stage_radix(L, NS);
    constexpr int P = fft_points(L);
    constexpr int TPS = fft_tps(L);
    constexpr int NB = P / R;
    constexpr int STRIDE = L / R;
    float2 v[P];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
#pragma unroll
      for (int j = 0; j < R; ++j) v[q * R + j] = s[pidx(t + j * STRIDE)];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
      const int k = t & (NS - 1);
      if constexpr (NS > 1) {
        const float2* twp = tw + tw_offset(L, NS) + k;
#pragma unroll
        for (int j = 1; j < R; ++j) {
          const float2 w = __ldg(twp + (j - 1) * NS);
          v[q * R + j] = INV ? cmulc(v[q * R + j], w) : cmul(v[q * R + j], w);
        }
      }
      dft<R, INV>(v + q * R);
      const int base = (t - k) * R + k;
#pragma unroll
      for (int m = 0; m < R; ++m) s[pidx(base + m * NS)] = v[q * R + m];
    }
    __syncthreads();
    fft_stages<L, NS * R, INV>(s, g, tw);
  }
}

// Whole FFT of length L (forward: e^{-2 pi i nk/L}; inverse: e^{+...}, unscaled).
template <int L, bool INV>
__device__ __forceinline__ void cta_fft(float2* __restrict__ s, int g, const float2* __restrict__ tw) {
  fft_stages<L, 1, INV>(s, g, tw);
}

}  // namespace gbdct
