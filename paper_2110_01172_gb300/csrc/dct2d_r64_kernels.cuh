// dct2d_r64_kernels.cuh - 2D DCT-II / inverse passes on the radix-64 engine.
//
// Same method as dct2d_kernels.cuh (arXiv 2110.01172, Algorithm 2 with the
// fused pre/postprocess of Section III), arranged so that each FFT makes as
// few shared-memory exchanges as possible (one for L = 4096):
//
//  * a CTA runs two sequences; lanes alternate between them (sequence s =
//    lane & 1, position t = lane >> 1), so the two lanes of a pair touch
//    neighbouring addresses in every global access;
//  * forward, column pass: the real-pair split of the column spectra is NOT
//    done here; the raw spectrum Z_p(k1) = DFT(v(:,p) + i v(:,N2-1-p)) is
//    stored column-pair-major (float4 (Z_2q(k1), Z_2q+1(k1)) at q*N1 + k1),
//    written straight from the last stage's registers;
//  * forward, row pass: the split is folded into the loads (rows k1 and
//    N1-k1 of Z give V1(k1, .) = DFT_n1 of the reordered columns), then the
//    row FFT and the symmetric-pair postprocess of Eqs. four-elements / s-t,
//    four outputs per two spectrum values, written as float4;
//  * inverse, row pass: the four-read preprocess of Eq. 2d_idct_pre is done
//    in the loads, the row FFT result U(k1, n2) is written row-pair-major
//    (float4 (U(k1,n2), U(k1+1,n2)) at (k1/2)*N2 + n2);
//  * inverse, column pass: Hermitian rebuild in the loads, column FFT, and
//    the inverse reorder of Eq. 2d_idct_post in the stores.
//
// Supported lengths: N1, N2 in {4096, 8192}.
#pragma once

#include "dct2d_kernels.cuh"
#include "fft_r64.cuh"

namespace gbdct {

template <int L>
struct R64Geom {
  static constexpr int TPS = r64::tps(L);
  static constexpr int THREADS = 2 * TPS;
  static constexpr int LP = r64::pad_len(L) + 8;  // +64 B: the two buffers start on different banks
  static constexpr size_t SMEM = 2 * (size_t)LP * sizeof(float2);
  static constexpr int R1 = r64::radix(L, 1);
  static constexpr int ST1 = L / R1;
  static constexpr int NSL = r64::last_ns(L);
  static constexpr int RL = r64::radix(L, NSL);
  static constexpr int NBL = r64::points(L) / RL;
};

// ----------------------------------------------------------------------------
// Forward, column pass (L = N1): reorder + FFT along n1 -> raw column spectra
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_fwd_cols_r64(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int N2 = a.n2;
  const int p = 2 * blockIdx.x + s;  // complex column = input columns (2p, 2p+1)
  const float* x = a.in + (long long)blockIdx.y * a.in_bstride;
  float2* Z = a.work + (long long)blockIdx.y * a.work_bstride;  // float2 index 2*(q*N1 + k1) + half

  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int r = reorder_src(t + j * G::ST1, L);
    v[j] = __ldg(reinterpret_cast<const float2*>(x + (long long)r * N2 + 2 * p));
  }
  r64::first_stage<L, false>(v, buf, t);
  __syncthreads();
  r64::stages_to_regs<L, G::R1, false>(buf, t, a.tw1, v);
  float2* Zq = Z + 2 * (long long)blockIdx.x * L + s;
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) Zq[2 * r64::out_pos<L>(t, qb, m)] = v[qb * G::RL + m];
}

// ----------------------------------------------------------------------------
// Forward, row pass (L = N2): split in the loads, row FFT, postprocess
// ----------------------------------------------------------------------------
// CTA b handles workspace rows k1 = 2b + s.  Row k1 >= 1 gives output rows k1
// and N1-k1; row 0 carries V1(0, .) + i V1(N1/2, .) and gives rows 0 and N1/2.
template <int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_fwd_rows_r64(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int N1 = a.n1;
  const int k1 = 2 * blockIdx.x + s;
  const bool packed = (k1 == 0);
  const int kmir = packed ? N1 / 2 : N1 - k1;
  const float2* Z = a.work + (long long)blockIdx.y * a.work_bstride;
  float* y = a.out + (long long)blockIdx.y * a.out_bstride;

  // V1(k1, n2) for the reordered column n2: column p = n2 (n2 < L/2) holds
  // Z_p = U + i Wt of columns p and L-1-p; U(k1) = (Z(k1) + conj Z(N1-k1))/2,
  // Wt(k1) = (Z(k1) - conj Z(N1-k1))/(2i).  Rows 0 and N1/2 are real.
  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int n2 = t + j * G::ST1;
    const bool lowhalf = n2 < L / 2;
    const int p = lowhalf ? n2 : L - 1 - n2;
    const long long base = 2 * ((long long)(p >> 1) * N1) + (p & 1);
    const float2 za = Z[base + 2 * k1];
    const float2 zb = Z[base + 2 * kmir];
    if (packed) {
      v[j] = lowhalf ? make_float2(za.x, zb.x) : make_float2(za.y, zb.y);
    } else {
      v[j] = lowhalf ? make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y))
                     : make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
    }
  }
  r64::first_stage<L, false>(v, buf, t);
  __syncthreads();
  r64::stages_to_regs<L, G::R1, false>(buf, t, a.tw2, v);
  // exchange: the postprocess pairs column k2 with L - k2
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) buf[r64::pidx(r64::out_pos<L>(t, qb, m))] = v[qb * G::RL + m];
  __syncthreads();

  const float2 av = __ldg(a.fa + k1);
  float* row0 = y + (long long)k1 * L;     // row k1 (0 for the packed row)
  float* row1 = y + (long long)kmir * L;   // row N1-k1 (N1/2 for the packed row)
  constexpr float RH = 0.70710678118654752f;
  // Quad pair i: columns Q = 4i..4i+3 and Q' = L-4i-4..L-4i-1.  Columns
  // 4i+d and L-4i-d (d = 1..3) are symmetric pairs: four outputs from s, t.
  // Columns 4i and L-4i-4 pair with columns of other quads: two outputs each.
  for (int i = t; i < L / 8; i += G::TPS) {
    const int c = 4 * i;
    float2 Yq[5], Ym[5];  // Yq[d] = Y(c+d), Ym[d] = Y((L-c-d) mod L)
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      Yq[d] = buf[r64::pidx(c + d)];
      Ym[d] = buf[r64::pidx((L - c - d) & (L - 1))];
    }
    float q0[4], q1[4], r0[4], r1[4];  // Q row0, Q row1, Q' row0, Q' row1 (ascending columns)
    // full symmetric pairs (c+d, L-c-d), d = 1..3 ; Q' index of L-c-d is 3-(d-1)... = 4-d
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      if (d >= 1 && d <= 3) {
        const float2 bt = __ldg(a.fb + c + d);
        const float2 P = Yq[d], M = Ym[d];
        if (packed) {
          const float2 sm0 = make_float2(P.x + M.x, P.y - M.y);                 // 2 V(0)
          const float2 dh = make_float2(RH * (P.y + M.y), RH * (M.x - P.x));    // sqrt2 V(N1/2)
          const float2 s0 = cmul(bt, sm0), sh = cmul(bt, dh);
          q0[d] = s0.x;
          q1[d] = sh.x;
          r0[4 - d] = -s0.y;
          r1[4 - d] = -sh.y;
        } else {
          const float2 aP = cmul(P, av);
          const float2 aM = cmul(M, av);
          const float2 u = make_float2(aP.x + aM.x, aP.y - aM.y);  // aP + conj(a) conj(M)
          const float2 w = make_float2(aP.x - aM.x, aP.y + aM.y);  // aP - conj(a) conj(M)
          const float2 sv = cmul(bt, u), tv = cmul(bt, w);
          q0[d] = sv.x;
          q1[d] = -tv.y;
          r0[4 - d] = -sv.y;
          r1[4 - d] = -tv.x;
        }
      }
    }
    // single columns: c (partner L-c) and L-c-4 (partner c+4)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = e ? (L - c - 4) : c;
      const float2 P = e ? Ym[4] : Yq[0];
      const float2 M = e ? Yq[4] : Ym[0];
      const float2 bt = __ldg(a.fb + col);
      float o0, o1;
      if (packed) {
        const float2 s0 = cmul(bt, make_float2(P.x + M.x, P.y - M.y));
        const float2 sh = cmul(bt, make_float2(RH * (P.y + M.y), RH * (M.x - P.x)));
        o0 = s0.x;
        o1 = sh.x;
      } else {
        const float2 aP = cmul(P, av);
        const float2 aM = cmul(M, av);
        const float2 u = make_float2(aP.x + aM.x, aP.y - aM.y);
        const float2 w = make_float2(aP.x - aM.x, aP.y + aM.y);
        o0 = bt.x * u.x - bt.y * u.y;
        o1 = -(bt.x * w.y + bt.y * w.x);
      }
      if (e) { r0[0] = o0; r1[0] = o1; } else { q0[0] = o0; q1[0] = o1; }
    }
    *reinterpret_cast<float4*>(row0 + c) = make_float4(q0[0], q0[1], q0[2], q0[3]);
    *reinterpret_cast<float4*>(row1 + c) = make_float4(q1[0], q1[1], q1[2], q1[3]);
    *reinterpret_cast<float4*>(row0 + L - c - 4) = make_float4(r0[0], r0[1], r0[2], r0[3]);
    *reinterpret_cast<float4*>(row1 + L - c - 4) = make_float4(r1[0], r1[1], r1[2], r1[3]);
  }
}

// ----------------------------------------------------------------------------
// Inverse, row pass (L = N2): four-read preprocess in the loads + row IFFT
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_inv_rows_r64(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int N1 = a.n1;
  const int k1 = 2 * blockIdx.x + s;
  const bool packed = (k1 == 0);
  const int kmir = packed ? N1 / 2 : N1 - k1;
  const float* C = a.in + (long long)blockIdx.y * a.in_bstride;
  const float* ca = C + (long long)k1 * L;
  const float* cb = C + (long long)kmir * L;
  float2* U = a.work + (long long)blockIdx.y * a.work_bstride;
  const float2 ia = __ldg(a.ia + k1);
  const float2 ih = __ldg(a.ia + N1 / 2);

  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int k2 = t + j * G::ST1;
    const int km = (L - k2) & (L - 1);
    const float c1 = __ldg(ca + k2), c3 = __ldg(cb + k2);
    const float c4 = k2 ? __ldg(ca + km) : 0.f;  // C(., N2) = 0
    const float c2 = k2 ? __ldg(cb + km) : 0.f;
    const float2 bk = __ldg(a.ib + k2);
    if (packed) {
      // V(0,k2) = a0 b [C(0,k2) - i C(0,N2-k2)];
      // V(h,k2) = ah b [(C(h,k2) - C(h,N2-k2)) - i (C(h,k2) + C(h,N2-k2))]
      const float2 v0 = cmul(cmul(make_float2(c1, -c4), bk), ia);
      const float2 vh = cmul(cmul(make_float2(c3 - c2, -(c3 + c2)), bk), ih);
      v[j] = make_float2(v0.x - vh.y, v0.y + vh.x);
    } else {
      v[j] = cmul(cmul(make_float2(c1 - c2, -(c3 + c4)), bk), ia);
    }
  }
  r64::first_stage<L, true>(v, buf, t);
  __syncthreads();
  r64::stages_to_regs<L, G::R1, true>(buf, t, a.tw2, v);
  float2* Ur = U + 2 * (long long)blockIdx.x * L + s;
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) Ur[2 * r64::out_pos<L>(t, qb, m)] = v[qb * G::RL + m];
}

// ----------------------------------------------------------------------------
// Inverse, column pass (L = N1): Hermitian rebuild + column IFFT + un-reorder
// ----------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_inv_cols_r64(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int N2 = a.n2;
  const int p = 2 * blockIdx.x + s;
  const int pq = N2 - 1 - p;
  const float2* U = a.work + (long long)blockIdx.y * a.work_bstride;  // 2*((k/2)*N2 + col) + (k&1)
  float* x = a.out + (long long)blockIdx.y * a.out_bstride;

  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int k1 = t + j * G::ST1;
    const bool upper = k1 > L / 2;
    const int kr = (k1 == L / 2) ? 0 : (upper ? L - k1 : k1);
    const long long rb = 2 * ((long long)(kr >> 1) * N2) + (kr & 1);
    const float2 wp = U[rb + 2 * p];
    const float2 wq = U[rb + 2 * pq];
    float2 z;
    if (k1 == 0) z = make_float2(wp.x, wq.x);
    else if (k1 == L / 2) z = make_float2(wp.y, wq.y);
    else if (!upper) z = make_float2(wp.x - wq.y, wp.y + wq.x);   // U(k,p) + i U(k,pq)
    else z = make_float2(wp.x + wq.y, wq.x - wp.y);               // conj U(k,p) + i conj U(k,pq)
    v[j] = z;
  }
  r64::first_stage<L, true>(v, buf, t);
  __syncthreads();
  r64::stages_to_regs<L, G::R1, true>(buf, t, a.tw1, v);
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) {
      const int n = r64::out_pos<L>(t, qb, m);
      *reinterpret_cast<float2*>(x + (long long)reorder_src(n, L) * N2 + 2 * p) = v[qb * G::RL + m];
    }
}

}  // namespace gbdct
