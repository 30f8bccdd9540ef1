// fft_core.cuh - CTA-level complex FFTs in shared memory (sm_103a).
//
// The FFT stage of the three-stage method (arXiv 2110.01172, Algorithm 2,
// "2D_RFFT") is computed here by hand-written radix-16/8/4/2 Stockham stages
// instead of a vendor library.  A sequence of length L = 16^a * r lives in
// shared memory; every thread keeps P = min(L, 16) points in registers during
// a stage, so one stage is: gather P points, multiply by the stage twiddles,
// run radix-R DFTs in registers, scatter the results back in autosorted
// (natural) order.  The radix-r stage, if any, comes last.
//
// Two element types are supported: float2 (one complex sequence) and float4
// (two independent complex sequences interleaved point by point, so every
// shared-memory access is 128-bit and every twiddle serves two sequences).
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

// Stage structure for at most `pmax` points per thread: L = pmax^a * r, radix
// pmax stages first, the radix-r stage (r < pmax) last.
__host__ __device__ constexpr int stage_radix_p(int L, int ns, int pmax) {
  return (L / ns >= pmax) ? pmax : (L / ns);
}
// Offset (in float2) of the twiddle block of the stage that starts at `ns`.
__host__ __device__ constexpr int tw_offset_p(int L, int ns, int pmax) {
  int off = 0;
  for (int n = 1; n < ns; n *= stage_radix_p(L, n, pmax)) {
    if (n > 1) off += (stage_radix_p(L, n, pmax) - 1) * n;
  }
  return off;
}
__host__ __device__ constexpr int tw_size_p(int L, int pmax) { return tw_offset_p(L, L, pmax); }

__host__ __device__ constexpr int fft_points(int L) { return L >= 16 ? 16 : L; }
__host__ __device__ constexpr int fft_tps(int L) { return L / fft_points(L); }
__host__ __device__ constexpr int stage_radix(int L, int ns) { return stage_radix_p(L, ns, 16); }
__host__ __device__ constexpr int tw_offset(int L, int ns) { return tw_offset_p(L, ns, 16); }
__host__ __device__ constexpr int tw_size(int L) { return tw_size_p(L, 16); }

// Padded shared-memory layouts.  The first stage writes each thread's 16
// outputs contiguously; the padding spreads those rows over all banks.
//   float2 elements: two float2 of padding after every 16 (keeps float4 pairs aligned)
//   float4 elements: one float4 of padding after every 16
template <typename T>
__host__ __device__ constexpr int pad_len(int L) {
  return (L < 16) ? L : (sizeof(T) == 8 ? L + (L >> 3) : L + (L >> 4));
}
template <typename T>
__device__ __forceinline__ int pidx(int i) {
  return (sizeof(T) == 8) ? i + ((i >> 4) << 1) : i + (i >> 4);
}

// ----------------------------------------------------------------------------
// Complex arithmetic on float2 (re, im) and float4 (re0, im0, re1, im1)
// ----------------------------------------------------------------------------

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 csub(float4 a, float4 b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float4 cmul(float4 a, float2 w) {
  return make_float4(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x),
                     fmaf(a.z, w.x, -a.w * w.y), fmaf(a.z, w.y, a.w * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
__device__ __forceinline__ float4 cmulc(float4 a, float2 w) {
  return make_float4(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y),
                     fmaf(a.z, w.x, a.w * w.y), fmaf(a.w, w.x, -a.z * w.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 lo(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Multiply by e^{-i pi/2} (forward) or e^{+i pi/2} (inverse).
template <bool INV>
__device__ __forceinline__ float2 mul_mj(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
template <bool INV>
__device__ __forceinline__ float4 mul_mj(float4 a) {
  return INV ? make_float4(-a.y, a.x, -a.w, a.z) : make_float4(a.y, -a.x, a.w, -a.z);
}

// a * (cr + i ci) for compile-time constants
__device__ __forceinline__ float2 cmulk(float2 a, float cr, float ci) {
  return make_float2(fmaf(cr, a.x, -ci * a.y), fmaf(cr, a.y, ci * a.x));
}
__device__ __forceinline__ float4 cmulk(float4 a, float cr, float ci) {
  return make_float4(fmaf(cr, a.x, -ci * a.y), fmaf(cr, a.y, ci * a.x),
                     fmaf(cr, a.z, -ci * a.w), fmaf(cr, a.w, ci * a.z));
}
// a * (c (1 + i s)) with c = +-sqrt(1/2), s = +-1: 2 adds and 2 multiplies
__device__ __forceinline__ float2 cmul_diag(float2 a, float c, float s) {
  return make_float2(c * (a.x - s * a.y), c * (a.y + s * a.x));
}
__device__ __forceinline__ float4 cmul_diag(float4 a, float c, float s) {
  return make_float4(c * (a.x - s * a.y), c * (a.y + s * a.x), c * (a.z - s * a.w), c * (a.w + s * a.z));
}
template <typename T>
__device__ __forceinline__ T cneg(T a);
template <>
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
template <>
__device__ __forceinline__ float4 cneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

// Multiply by W16^E = exp(-+ 2 pi i E / 16) for a compile-time E.
template <int E, bool INV, typename T>
__device__ __forceinline__ T mul_w16(T a) {
  constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
  constexpr float RH = 0.70710678118654752f;  // sqrt(1/2)
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return mul_mj<INV>(a);
  } else if constexpr (e == 8) {
    return cneg(a);
  } else if constexpr (e == 12) {
    return mul_mj<!INV>(a);
  } else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
    // e pi / 8 is an odd multiple of pi/4: twiddle (cr + i ci) with |cr| = |ci|
    constexpr float cr = (e == 2 || e == 14) ? RH : -RH;
    constexpr float ci0 = (e == 2 || e == 6) ? -RH : RH;  // forward imaginary part
    constexpr float ci = INV ? -ci0 : ci0;
    return cmul_diag(a, cr, ci / cr);
  } else {
    constexpr int q = e & 3;  // 1 or 3
    constexpr float c0 = (q == 1) ? C1 : S1;
    constexpr float s0 = (q == 1) ? S1 : C1;
    constexpr int quad = e >> 2;
    constexpr float cs = (quad == 0) ? c0 : (quad == 1) ? -s0 : (quad == 2) ? -c0 : s0;
    constexpr float sn = (quad == 0) ? s0 : (quad == 1) ? c0 : (quad == 2) ? -s0 : -c0;
    // forward twiddle = cos - i sin; inverse = cos + i sin
    return cmulk(a, cs, INV ? sn : -sn);
  }
}

// ----------------------------------------------------------------------------
// Radix-R DFTs in registers (X_m = sum_j a_j W_R^{jm}, W_R = e^{-+2 pi i/R})
// ----------------------------------------------------------------------------

template <bool INV, typename T>
__device__ __forceinline__ void dft4(T& a0, T& a1, T& a2, T& a3) {
  const T t0 = cadd(a0, a2), t1 = csub(a0, a2);
  const T t2 = cadd(a1, a3), t3 = mul_mj<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(T* v) {
  if constexpr (R == 2) {
    const T t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // 8 = 2 x 4: DFT4 of even and odd points, twiddle W8^k, radix-2 combine
    T e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    T o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_w16<2, INV>(o1);
    o2 = mul_w16<4, INV>(o2);
    o3 = mul_w16<6, INV>(o3);
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
  } else if constexpr (R == 16) {
    // 16 = 4 x 4: DFT4s over n1 (stride 4), twiddles W16^{n2 k1}, DFT4s over n2
    dft4<INV>(v[0], v[4], v[8], v[12]);
    dft4<INV>(v[1], v[5], v[9], v[13]);
    dft4<INV>(v[2], v[6], v[10], v[14]);
    dft4<INV>(v[3], v[7], v[11], v[15]);
    v[5] = mul_w16<1, INV>(v[5]);
    v[9] = mul_w16<2, INV>(v[9]);
    v[13] = mul_w16<3, INV>(v[13]);
    v[6] = mul_w16<2, INV>(v[6]);
    v[10] = mul_w16<4, INV>(v[10]);
    v[14] = mul_w16<6, INV>(v[14]);
    v[7] = mul_w16<3, INV>(v[7]);
    v[11] = mul_w16<6, INV>(v[11]);
    v[15] = mul_w16<9, INV>(v[15]);
    T t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      T a0 = v[4 * k1 + 0], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
      dft4<INV>(a0, a1, a2, a3);
      t[k1 + 0] = a0;
      t[k1 + 4] = a1;
      t[k1 + 8] = a2;
      t[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
  }
}

// ----------------------------------------------------------------------------
// Stockham stages
// ----------------------------------------------------------------------------

// Twiddle + radix-R DFT of butterfly t of the stage starting at NS, in place
// on the R registers at v.
template <int L, int NS, bool INV, typename T>
__device__ __forceinline__ void stage_butterfly(T* v, int t, const float2* __restrict__ tw) {
  constexpr int R = stage_radix(L, NS);
  if constexpr (NS > 1) {
    const int k = t & (NS - 1);
    const float2* twp = tw + tw_offset(L, NS) + k;
#pragma unroll
    for (int j = 1; j < R; ++j) {
      const float2 w = __ldg(twp + (j - 1) * NS);
      v[j] = INV ? cmulc(v[j], w) : cmul(v[j], w);
    }
  }
  dft<R, INV>(v);
}

// Destination index of output m of butterfly t in the stage starting at NS.
template <int L, int NS>
__device__ __forceinline__ int stage_out_index(int t, int m) {
  const int k = t & (NS - 1);
  return (t - k) * stage_radix(L, NS) + k + m * NS;
}

// Stages NS .. L on the sequence at `s` (padded layout, natural order in and
// out).  `g` in [0, fft_tps(L)) is the thread's rank within the sequence; every
// thread of the CTA must call this (it contains __syncthreads).
template <int L, int NS, bool INV, typename T>
__device__ __forceinline__ void fft_stages(T* __restrict__ s, int g, const float2* __restrict__ tw) {
  if constexpr (NS < L) {
    constexpr int R = stage_radix(L, NS);
    constexpr int P = fft_points(L);
    constexpr int TPS = fft_tps(L);
    constexpr int NB = P / R;
    constexpr int STRIDE = L / R;
    T v[P];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
#pragma unroll
      for (int j = 0; j < R; ++j) v[q * R + j] = s[pidx<T>(t + j * STRIDE)];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
      stage_butterfly<L, NS, INV>(v + q * R, t, tw);
#pragma unroll
      for (int m = 0; m < R; ++m) s[pidx<T>(stage_out_index<L, NS>(t, m))] = v[q * R + m];
    }
    __syncthreads();
    fft_stages<L, NS * R, INV>(s, g, tw);
  }
}

// Whole FFT of length L (forward: e^{-2 pi i nk/L}; inverse: e^{+...}, unscaled).
template <int L, bool INV, typename T>
__device__ __forceinline__ void cta_fft(T* __restrict__ s, int g, const float2* __restrict__ tw) {
  fft_stages<L, 1, INV>(s, g, tw);
}

// First stage from registers: v holds the points g + j * (L / R1) (j < R1) of
// the natural-order input; runs the first radix-R1 stage and stores to `s`.
// The caller synchronises before the next stage (fft_stages<L, R1>).
template <int L, bool INV, typename T>
__device__ __forceinline__ void first_stage_regs(T* v, T* __restrict__ s, int g) {
  constexpr int R = stage_radix(L, 1);
  dft<R, INV>(v);
#pragma unroll
  for (int m = 0; m < R; ++m) s[pidx<T>(g * R + m)] = v[m];
}

// Stages NS .. L where the last stage leaves its outputs in registers instead
// of shared memory.  On return, for L >= 16 with a radix-16 last stage, thread
// g holds outputs at positions g + m * (L/16) (m < 16) in v; in general it
// holds NB butterflies: output (q, m) is at stage_out_index<L, NSlast>(g + q*TPS, m).
// Requires at least two stages remaining (NS < L).
template <int L, int NS, bool INV, typename T>
__device__ __forceinline__ void fft_stages_to_regs(T* __restrict__ s, int g, const float2* __restrict__ tw,
                                                   T* v) {
  constexpr int R = stage_radix(L, NS);
  constexpr int P = fft_points(L);
  constexpr int TPS = fft_tps(L);
  constexpr int NB = P / R;
  constexpr int STRIDE = L / R;
  if constexpr (NS * R < L) {
    fft_stages<L, NS, INV>(s, g, tw);  // unreachable by construction; keeps the template total
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
#pragma unroll
      for (int j = 0; j < R; ++j) v[q * R + j] = s[pidx<T>(t + j * STRIDE)];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) stage_butterfly<L, NS, INV>(v + q * R, g + q * TPS, tw);
  }
}

// The start of the last stage of a length-L FFT.
__host__ __device__ constexpr int last_stage_ns(int L) {
  int n = 1;
  while (n * stage_radix(L, n) < L) n *= stage_radix(L, n);
  return n;
}

// Runs every stage from NS up to (but excluding) the last one through shared
// memory, then the last stage into registers (see fft_stages_to_regs).
template <int L, int NS, bool INV, typename T>
__device__ __forceinline__ void fft_stages_last_regs(T* __restrict__ s, int g, const float2* __restrict__ tw,
                                                     T* v) {
  constexpr int NL = last_stage_ns(L);
  if constexpr (NS < NL) {
    constexpr int R = stage_radix(L, NS);
    constexpr int P = fft_points(L);
    constexpr int TPS = fft_tps(L);
    constexpr int NB = P / R;
    constexpr int STRIDE = L / R;
    T w[P];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
#pragma unroll
      for (int j = 0; j < R; ++j) w[q * R + j] = s[pidx<T>(t + j * STRIDE)];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
      stage_butterfly<L, NS, INV>(w + q * R, t, tw);
#pragma unroll
      for (int m = 0; m < R; ++m) s[pidx<T>(stage_out_index<L, NS>(t, m))] = w[q * R + m];
    }
    __syncthreads();
    fft_stages_last_regs<L, NS * R, INV>(s, g, tw, v);
  } else {
    fft_stages_to_regs<L, NL, INV>(s, g, tw, v);
  }
}

}  // namespace gbdct
