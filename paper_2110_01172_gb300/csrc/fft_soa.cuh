// fft_soa.cuh - radix-16 Stockham FFT on two sequences at once, in packed
// two-lane FP32 arithmetic (sm_100+ add/mul/fma .f32x2).
//
// A value of type C2 holds the same point of two independent complex
// sequences in structure-of-arrays form: re = (re_a, re_b), im = (im_a, im_b).
// Both sequences follow the same data flow with the same twiddles, so every
// complex add is two packed adds and every complex multiply four packed
// multiply/fma instructions, half the instruction count of the one-sequence
// engine in fft_core.cuh for the same arithmetic.  The radix-16 DFT is 4 x 4
// (DFT4s, internal twiddles W16^{n2 k1}, DFT4s), as in fft_core.cuh.
//
// Shared memory holds one float4 (re_a, re_b, im_a, im_b) per point, with one
// float4 of padding after every 16 (pidx<float4>), so a stage's per-thread
// runs of 16 outputs fall on distinct banks.  Stage twiddles come from a float4
// table (wr, wr, wi, wi) with the index layout of fft_core.cuh's float2 table.
#pragma once

#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace gbdct {
namespace soa {

struct C2 {
  float2 re, im;
};

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 ng(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, ng(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ C2 add(C2 a, C2 b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ C2 sub(C2 a, C2 b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }

// a * (wr + i wi); wr, wi are lane pairs (the same or different per lane)
__device__ __forceinline__ C2 mulw(C2 a, float2 wr, float2 wi) {
  return {fma2(a.im, ng(wi), mul2(a.re, wr)), fma2(a.im, wr, mul2(a.re, wi))};
}
// a * conj(wr + i wi)
__device__ __forceinline__ C2 mulwc(C2 a, float2 wr, float2 wi) {
  return {fma2(a.im, wi, mul2(a.re, wr)), fma2(a.re, ng(wi), mul2(a.im, wr))};
}
// a * (-i) forward, a * (+i) inverse
template <bool INV>
__device__ __forceinline__ C2 mul_mj(C2 a) {
  return INV ? C2{ng(a.im), a.re} : C2{a.im, ng(a.re)};
}

__device__ __forceinline__ float4 pack(C2 a) { return make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }
// The two points as two interleaved complex values (re_a, im_a, re_b, im_b),
// the layout of a pair of adjacent complex columns in global memory.
__device__ __forceinline__ float4 pack_aos(C2 a) { return make_float4(a.re.x, a.im.x, a.re.y, a.im.y); }
__device__ __forceinline__ C2 unpack(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }

// Multiply by W16^E = exp(-+2 pi i E / 16) for a compile-time E.
template <int E, bool INV>
__device__ __forceinline__ C2 mul_w16(C2 a) {
  constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
  constexpr float RH = 0.70710678118654752f;  // sqrt(1/2)
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 4) {
    return mul_mj<INV>(a);
  } else if constexpr (e == 8) {
    return C2{ng(a.re), ng(a.im)};
  } else if constexpr (e == 12) {
    return mul_mj<!INV>(a);
  } else if constexpr (e == 2 || e == 6 || e == 10 || e == 14) {
    // odd multiple of pi/4: c (1 + i s) with |c| = sqrt(1/2), s = +-1
    constexpr float cr = (e == 2 || e == 14) ? RH : -RH;
    constexpr float ci0 = (e == 2 || e == 6) ? -RH : RH;  // forward imaginary part
    constexpr float ci = INV ? -ci0 : ci0;
    // re' = cr re - ci im, im' = cr im + ci re
    return C2{fma2(a.im, bc(-ci), mul2(a.re, bc(cr))), fma2(a.re, bc(ci), mul2(a.im, bc(cr)))};
  } else {
    constexpr int q = e & 3;
    constexpr float c0 = (q == 1) ? C1 : S1;
    constexpr float s0 = (q == 1) ? S1 : C1;
    constexpr int quad = e >> 2;
    constexpr float cs = (quad == 0) ? c0 : (quad == 1) ? -s0 : (quad == 2) ? -c0 : s0;
    constexpr float sn = (quad == 0) ? s0 : (quad == 1) ? c0 : (quad == 2) ? -s0 : -c0;
    constexpr float ci = INV ? sn : -sn;
    return C2{fma2(a.im, bc(-ci), mul2(a.re, bc(cs))), fma2(a.re, bc(ci), mul2(a.im, bc(cs)))};
  }
}

template <bool INV>
__device__ __forceinline__ void dft4(C2& a0, C2& a1, C2& a2, C2& a3) {
  const C2 t0 = add(a0, a2), t1 = sub(a0, a2);
  const C2 t2 = add(a1, a3), d = sub(a1, a3);
  a0 = add(t0, t2);
  a2 = sub(t0, t2);
  if constexpr (!INV) {  // t3 = -i d
    a1 = C2{add2(t1.re, d.im), sub2(t1.im, d.re)};
    a3 = C2{sub2(t1.re, d.im), add2(t1.im, d.re)};
  } else {  // t3 = +i d
    a1 = C2{sub2(t1.re, d.im), add2(t1.im, d.re)};
    a3 = C2{add2(t1.re, d.im), sub2(t1.im, d.re)};
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(C2* v) {
  if constexpr (R == 2) {
    const C2 t = v[0];
    v[0] = add(t, v[1]);
    v[1] = sub(t, v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    C2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_w16<2, INV>(o1);
    o2 = mul_w16<4, INV>(o2);
    o3 = mul_w16<6, INV>(o3);
    v[0] = add(e0, o0); v[4] = sub(e0, o0);
    v[1] = add(e1, o1); v[5] = sub(e1, o1);
    v[2] = add(e2, o2); v[6] = sub(e2, o2);
    v[3] = add(e3, o3); v[7] = sub(e3, o3);
  } else if constexpr (R == 16) {
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
    C2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C2 a0 = v[4 * k1 + 0], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
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

__device__ __forceinline__ int pidx4(int i) { return i + (i >> 4); }

__device__ __forceinline__ C2 ldw(const float4* p) {
  const float4 w = __ldg(p);
  return C2{make_float2(w.x, w.y), make_float2(w.z, w.w)};
}
__device__ __forceinline__ C2 wmul(C2 a, C2 b) { return mulw(a, b.re, b.im); }
template <bool INV>
__device__ __forceinline__ C2 apply(C2 u, C2 w) {
  return INV ? mulwc(u, w.re, w.im) : mulw(u, w.re, w.im);
}

// u[j] *= w^j (conjugated for the inverse), j = 1 .. R-1, where entry (j-1)*NS
// of twp is w^j.  Only the power-of-two powers are read (w, w^2, w^4, w^8 for
// R = 16); the other powers are products of at most three of them (a few ulp
// from the exactly rounded values), which keeps the table reads (and
// registers) low.
template <int R, bool INV>
__device__ __forceinline__ void twiddle(C2* u, const float4* __restrict__ twp, int NS) {
  if constexpr (R == 16) {
    const C2 w1 = ldw(twp), w2 = ldw(twp + NS), w4 = ldw(twp + 3 * NS), w8 = ldw(twp + 7 * NS);
    const C2 w3 = wmul(w1, w2);
    u[1] = apply<INV>(u[1], w1);
    u[2] = apply<INV>(u[2], w2);
    u[3] = apply<INV>(u[3], w3);
    u[4] = apply<INV>(u[4], w4);
    u[5] = apply<INV>(u[5], wmul(w1, w4));
    u[6] = apply<INV>(u[6], wmul(w2, w4));
    const C2 w7 = wmul(w3, w4);
    u[7] = apply<INV>(u[7], w7);
    u[8] = apply<INV>(u[8], w8);
    u[9] = apply<INV>(u[9], wmul(w1, w8));
    u[10] = apply<INV>(u[10], wmul(w2, w8));
    u[11] = apply<INV>(u[11], wmul(w3, w8));
    const C2 w12 = wmul(w4, w8);
    u[12] = apply<INV>(u[12], w12);
    u[13] = apply<INV>(u[13], wmul(w1, w12));
    u[14] = apply<INV>(u[14], wmul(w2, w12));
    u[15] = apply<INV>(u[15], wmul(w7, w8));
  } else if constexpr (R == 8) {  // w, w^2, w^4 read; the rest are their products
    const C2 w1 = ldw(twp), w2 = ldw(twp + NS), w4 = ldw(twp + 3 * NS);
    const C2 w3 = wmul(w1, w2);
    u[1] = apply<INV>(u[1], w1);
    u[2] = apply<INV>(u[2], w2);
    u[3] = apply<INV>(u[3], w3);
    u[4] = apply<INV>(u[4], w4);
    u[5] = apply<INV>(u[5], wmul(w1, w4));
    u[6] = apply<INV>(u[6], wmul(w2, w4));
    u[7] = apply<INV>(u[7], wmul(w3, w4));
  } else if constexpr (R == 4) {
    const C2 w1 = ldw(twp), w2 = ldw(twp + NS);
    u[1] = apply<INV>(u[1], w1);
    u[2] = apply<INV>(u[2], w2);
    u[3] = apply<INV>(u[3], wmul(w1, w2));
  } else {
#pragma unroll
    for (int j = 1; j < R; ++j) u[j] = apply<INV>(u[j], ldw(twp + (j - 1) * NS));
  }
}

// First stage from registers: v holds points g + j (L/16) of both sequences;
// radix-16 DFT, outputs g*16 + m stored to s.  Point i of the sequence pair
// lives at s[ST * pidx4(i)]: ST > 1 interleaves ST sequence pairs point by
// point (the column passes of the two-pass family, whose warps span pairs).
template <int L, bool INV, int ST = 1>
__device__ __forceinline__ void first_stage(C2* v, float4* __restrict__ s, int g) {
  constexpr int R = stage_radix(L, 1);
  dft<R, INV>(v);
#pragma unroll
  for (int m = 0; m < R; ++m) s[ST * pidx4(g * R + m)] = pack(v[m]);
}

// Shared-memory slot of output point k of the last stage: OUT = 0 the padded
// layout (pidx4), OUT = 1 dense (k), OUT = 2 dense with the upper half
// reversed (L/2 + (L-1-k) for k >= L/2), the order in which a bulk tensor
// store writes the rows of the two reorder residues.  Consecutive k of a
// stage's last writes stay on distinct banks in all three.  The dense forms
// are read by bulk tensor stores, so their slots hold the global-memory
// layout (pack_aos) instead of the engine's two-lane layout (pack).
template <int L, int OUT>
__device__ __forceinline__ int out_slot(int k) {
  if constexpr (OUT == 0) return pidx4(k);
  else if constexpr (OUT == 1) return k;
  else return k < L / 2 ? k : (3 * L / 2 - 1 - k);
}

// Stages NS .. L through shared memory (natural order in and out); every
// thread of the CTA calls this (it contains __syncthreads).  The last stage
// writes its outputs at out_slot<L, OUT>.
template <int L, int NS, bool INV, int ST = 1, int OUT = 0>
__device__ __forceinline__ void stages(float4* __restrict__ s, int g, const float4* __restrict__ tw) {
  if constexpr (NS < L) {
    constexpr int R = stage_radix(L, NS);
    constexpr int P = fft_points(L);
    constexpr int TPS = fft_tps(L);
    constexpr int NB = P / R;
    constexpr int STRIDE = L / R;
    C2 v[P];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
#pragma unroll
      for (int j = 0; j < R; ++j) v[q * R + j] = unpack(s[ST * pidx4(t + j * STRIDE)]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int t = g + q * TPS;
      C2* u = v + q * R;
      const int k = t & (NS - 1);
      twiddle<R, INV>(u, tw + tw_offset(L, NS) + k, NS);
      dft<R, INV>(u);
      if constexpr (NS * R < L) {
#pragma unroll
        for (int m = 0; m < R; ++m) s[ST * pidx4(stage_out_index<L, NS>(t, m))] = pack(u[m]);
      } else {
#pragma unroll
        for (int m = 0; m < R; ++m)
          s[ST * out_slot<L, OUT>(stage_out_index<L, NS>(t, m))] = OUT ? pack_aos(u[m]) : pack(u[m]);
      }
    }
    __syncthreads();
    stages<L, NS * R, INV, ST, OUT>(s, g, tw);
  }
}

}  // namespace soa
}  // namespace gbdct
