// dct2d_pair_kernels.cuh - the four 2D passes on two interleaved sequences.
//
// Same method and data flow as dct2d_kernels.cuh (arXiv 2110.01172,
// Algorithm 2 with the fused pre/post of Section III), organised for sm_103a
// instruction efficiency:
//
//  * every thread works on a float4 that holds the same point of two
//    independent sequences, so each shared-memory access is 128-bit and every
//    stage twiddle is loaded once for two sequences;
//  * a CTA handles PB such pairs, PB chosen per length so that a CTA has 256
//    threads (512 at L = 8192);
//  * the first FFT stage reads its points straight from global memory (the
//    reorder of Eq. 2d_dct_pre is only an address computation), and the
//    inverse passes write their last stage straight from registers;
//  * the half-spectrum workspace is stored as row pairs: element (k, c) of
//    the N1/2 x N2 complex workspace is at float4 index (k/2)*N2 + c, half
//    k%2, so the column pass writes 32-byte chunks and the row pass reads
//    whole float4 rows.
//
// Geometry requirements: 16 <= N1, N2 <= 8192, powers of two.
#pragma once

#include "dct2d_kernels.cuh"

#ifndef GBDCT_PAIR_MINB
#define GBDCT_PAIR_MINB 2
#endif

namespace gbdct {

template <int L>
struct PairGeom {
  static constexpr int TPS = fft_tps(L);                      // threads per pair
  static constexpr int PB = (256 / TPS) > 0 ? (256 / TPS) : 1;  // pairs per CTA
  static constexpr int THREADS = PB * TPS;
  static constexpr int LP = pad_len<float4>(L);
  static constexpr size_t SMEM = (size_t)PB * LP * sizeof(float4);
  static constexpr int R1 = stage_radix(L, 1);
  static constexpr int ST1 = L / R1;
  static constexpr int MINB = (THREADS <= 256) ? GBDCT_PAIR_MINB : 1;  // resident CTAs per SM
};

// ----------------------------------------------------------------------------
// Forward, column pass: reorder + FFT along n1 of two complex columns + split
// ----------------------------------------------------------------------------
// Pair q = complex columns (2q, 2q+1) = input columns 4q..4q+3: one float4
// load per row gives both sequences' points (Eq. 2d_dct_pre: input column
// 2p is reordered column p, input column 2p+1 is reordered column N2-1-p).
template <int L>
__global__ void __launch_bounds__(PairGeom<L>::THREADS, PairGeom<L>::MINB)
k_fwd_cols2(Dct2dArgs a) {
  using G = PairGeom<L>;
  extern __shared__ float4 sm4[];
  const int tid = threadIdx.x;
  const int lp = tid / G::TPS, g = tid % G::TPS;
  const int N2 = a.n2;
  const int npairs = N2 >> 2;
  int q = blockIdx.x * G::PB + lp;
  const bool valid = q < npairs;
  if (!valid) q = npairs - 1;
  float4* s = sm4 + lp * G::LP;
  const float* x = a.in + (long long)blockIdx.y * a.in_bstride;
  float4* Wp = reinterpret_cast<float4*>(a.work + (long long)blockIdx.y * a.work_bstride);

  float4 v[G::R1];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int r = reorder_src(g + j * G::ST1, L);
    v[j] = __ldg(reinterpret_cast<const float4*>(x + (long long)r * N2) + q);
  }
  first_stage_regs<L, false>(v, s, g);
  __syncthreads();
  fft_stages<L, G::R1, false>(s, g, a.tw1);

  // Split Z = FFT(u + i w) of each sequence into U (column p) and Wt (column
  // N2-1-p):  U[k] = (Z[k] + conj Z[L-k]) / 2,  Wt[k] = (Z[k] - conj Z[L-k]) / (2i);
  // row 0 packs the real values at k = 0 and k = L/2.
  for (int kk = g; kk < L / 4; kk += G::TPS) {
    const int k = 2 * kk;
    const float4 zk = s[pidx<float4>(k)];
    const float4 zk1 = s[pidx<float4>(k + 1)];
    const float4 zm = s[pidx<float4>(k == 0 ? L / 2 : L - k)];
    const float4 zm1 = s[pidx<float4>(L - k - 1)];
    float2 u0[2], w0[2], u1[2], w1[2];  // [row k, row k+1] for sequences 0 and 1
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2 Zk = h ? hi(zk) : lo(zk), Zm = h ? hi(zm) : lo(zm);
      const float2 Zk1 = h ? hi(zk1) : lo(zk1), Zm1 = h ? hi(zm1) : lo(zm1);
      float2 uk, wk;
      if (k == 0) {
        uk = make_float2(Zk.x, Zm.x);
        wk = make_float2(Zk.y, Zm.y);
      } else {
        uk = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
        wk = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
      }
      const float2 uk1 = make_float2(0.5f * (Zk1.x + Zm1.x), 0.5f * (Zk1.y - Zm1.y));
      const float2 wk1 = make_float2(0.5f * (Zk1.y + Zm1.y), 0.5f * (Zm1.x - Zk1.x));
      if (h == 0) { u0[0] = uk; u0[1] = uk1; w0[0] = wk; w0[1] = wk1; }
      else { u1[0] = uk; u1[1] = uk1; w1[0] = wk; w1[1] = wk1; }
    }
    if (valid) {
      float4* row = Wp + (long long)kk * N2;
      row[2 * q] = pack2(u0[0], u0[1]);
      row[2 * q + 1] = pack2(u1[0], u1[1]);
      row[N2 - 1 - 2 * q] = pack2(w0[0], w0[1]);
      row[N2 - 2 - 2 * q] = pack2(w1[0], w1[1]);
    }
  }
}

// ----------------------------------------------------------------------------
// Forward, row pass: FFT along n2 of two workspace rows + postprocess
// ----------------------------------------------------------------------------
// Pair m = workspace rows (2m, 2m+1).  For row k1 >= 1 the outputs of rows k1
// and N1-k1 at every column k2 are (Section III-B, Eqs. four-elements, s-t)
//   y(k1, k2)    =  Re( b/2 (a P + conj(a) Q) )
//   y(N1-k1, k2) = -Im( b/2 (a P - conj(a) Q) ),  P = V(k1,k2), Q = conj V(k1, N2-k2);
// row 0 holds V(0, .) + i V(N1/2, .) and gives output rows 0 and N1/2.
template <int L>
__global__ void __launch_bounds__(PairGeom<L>::THREADS, PairGeom<L>::MINB)
k_fwd_rows2(Dct2dArgs a) {
  using G = PairGeom<L>;
  extern __shared__ float4 sm4[];
  const int tid = threadIdx.x;
  const int lp = tid / G::TPS, g = tid % G::TPS;
  const int N1 = a.n1;
  const int npairs = N1 >> 2;
  int m = blockIdx.x * G::PB + lp;
  const bool valid = m < npairs;
  if (!valid) m = npairs - 1;
  float4* s = sm4 + lp * G::LP;
  const float4* Wp = reinterpret_cast<const float4*>(a.work + (long long)blockIdx.y * a.work_bstride);
  float* y = a.out + (long long)blockIdx.y * a.out_bstride;

  float4 v[G::R1];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) v[j] = Wp[(long long)m * L + g + j * G::ST1];
  first_stage_regs<L, false>(v, s, g);
  __syncthreads();
  fft_stages<L, G::R1, false>(s, g, a.tw2);
  if (!valid) return;

  const int k1a = 2 * m, k1b = 2 * m + 1;
  const float2 fa_a = __ldg(a.fa + k1a);
  const float2 fa_b = __ldg(a.fa + k1b);
  float* ya0 = y + (long long)(k1a == 0 ? 0 : k1a) * L;
  float* ya1 = y + (long long)(k1a == 0 ? N1 / 2 : N1 - k1a) * L;
  float* yb0 = y + (long long)k1b * L;
  float* yb1 = y + (long long)(N1 - k1b) * L;
  constexpr float RH = 0.70710678118654752f;  // (a + conj a) / 2 at k1 = N1/2
  for (int c4 = g; c4 < L / 4; c4 += G::TPS) {
    const int c = 4 * c4;
    const float4 b01 = __ldg(reinterpret_cast<const float4*>(a.fb + c));      // b/2 at c, c+1
    const float4 b23 = __ldg(reinterpret_cast<const float4*>(a.fb + c) + 1);  // b/2 at c+2, c+3
    float oa0[4], oa1[4], ob0[4], ob1[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int k2 = c + d;
      const float2 bt = (d == 0) ? lo(b01) : (d == 1) ? hi(b01) : (d == 2) ? lo(b23) : hi(b23);
      const float4 Y = s[pidx<float4>(k2)];
      const float4 Ym = s[pidx<float4>((L - k2) & (L - 1))];
      // sequence a (row k1a)
      {
        const float2 P = lo(Y), Mq = lo(Ym);
        if (k1a == 0) {
          // 2 V(0,k2) = Y + conj Ym;  2 V(N1/2,k2) = (Y - conj Ym) / i
          const float2 s0 = make_float2(P.x + Mq.x, P.y - Mq.y);
          const float2 sh = make_float2(RH * (P.y + Mq.y), RH * (Mq.x - P.x));
          oa0[d] = bt.x * s0.x - bt.y * s0.y;
          oa1[d] = bt.x * sh.x - bt.y * sh.y;
        } else {
          const float2 aP = cmul(P, fa_a);
          const float2 aYm = cmul(Mq, fa_a);
          const float2 aQc = make_float2(aYm.x, -aYm.y);  // conj(a) Q = conj(a Ym), Q = conj Ym
          const float2 u = cadd(aP, aQc), w = csub(aP, aQc);
          oa0[d] = bt.x * u.x - bt.y * u.y;
          oa1[d] = -(bt.x * w.y + bt.y * w.x);
        }
      }
      // sequence b (row k1b >= 1)
      {
        const float2 P = hi(Y), Mq = hi(Ym);
        const float2 aP = cmul(P, fa_b);
        const float2 aYm = cmul(Mq, fa_b);
        const float2 aQc = make_float2(aYm.x, -aYm.y);  // conj(a) conj(Ym) = conj(a Ym)
        const float2 u = cadd(aP, aQc), w = csub(aP, aQc);
        ob0[d] = bt.x * u.x - bt.y * u.y;
        ob1[d] = -(bt.x * w.y + bt.y * w.x);
      }
    }
    *reinterpret_cast<float4*>(ya0 + c) = make_float4(oa0[0], oa0[1], oa0[2], oa0[3]);
    *reinterpret_cast<float4*>(ya1 + c) = make_float4(oa1[0], oa1[1], oa1[2], oa1[3]);
    *reinterpret_cast<float4*>(yb0 + c) = make_float4(ob0[0], ob0[1], ob0[2], ob0[3]);
    *reinterpret_cast<float4*>(yb1 + c) = make_float4(ob1[0], ob1[1], ob1[2], ob1[3]);
  }
}

// ----------------------------------------------------------------------------
// Inverse, row pass: four-read preprocess + inverse FFT along k2 -> workspace
// ----------------------------------------------------------------------------
// Pair m = workspace rows (2m, 2m+1).  Row k1 needs input rows k1 and N1-k1
// (row 0: rows 0 and N1/2).  The four rows are first staged in shared memory
// as float4 (one per column), then every point of the first FFT stage is built
// in registers from two such float4 (Eq. 2d_idct_pre, conjugated twiddle):
//   V(k1,k2) = conj(a_k1) conj(b_k2) [C(k1,k2) - C(N1-k1,N2-k2) - i(C(N1-k1,k2) + C(k1,N2-k2))]
// with C(., N2) = 0, and 1/(N1 N2) folded into the a-table.
template <int L>
__global__ void __launch_bounds__(PairGeom<L>::THREADS, PairGeom<L>::MINB)
k_inv_rows2(Dct2dArgs a) {
  using G = PairGeom<L>;
  extern __shared__ float4 sm4[];
  const int tid = threadIdx.x;
  const int lp = tid / G::TPS, g = tid % G::TPS;
  const int N1 = a.n1;
  const int npairs = N1 >> 2;
  int m = blockIdx.x * G::PB + lp;
  const bool valid = m < npairs;
  if (!valid) m = npairs - 1;
  float4* s = sm4 + lp * G::LP;
  const float* C = a.in + (long long)blockIdx.y * a.in_bstride;
  float4* Wp = reinterpret_cast<float4*>(a.work + (long long)blockIdx.y * a.work_bstride);

  const int k1a = 2 * m, k1b = 2 * m + 1;
  const float* ra = C + (long long)k1a * L;
  const float* rb = C + (long long)(k1a == 0 ? N1 / 2 : N1 - k1a) * L;
  const float* rc = C + (long long)k1b * L;
  const float* rd = C + (long long)(N1 - k1b) * L;
  for (int c4 = g; c4 < L / 4; c4 += G::TPS) {
    const float4 A = __ldg(reinterpret_cast<const float4*>(ra) + c4);
    const float4 B = __ldg(reinterpret_cast<const float4*>(rb) + c4);
    const float4 Cc = __ldg(reinterpret_cast<const float4*>(rc) + c4);
    const float4 D = __ldg(reinterpret_cast<const float4*>(rd) + c4);
    const int c = 4 * c4;
    s[pidx<float4>(c + 0)] = make_float4(A.x, B.x, Cc.x, D.x);
    s[pidx<float4>(c + 1)] = make_float4(A.y, B.y, Cc.y, D.y);
    s[pidx<float4>(c + 2)] = make_float4(A.z, B.z, Cc.z, D.z);
    s[pidx<float4>(c + 3)] = make_float4(A.w, B.w, Cc.w, D.w);
  }
  __syncthreads();

  const float2 ia_a = __ldg(a.ia + k1a);
  const float2 ia_h = __ldg(a.ia + N1 / 2);
  const float2 ia_b = __ldg(a.ia + k1b);
  float4 v[fft_points(L)];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int k2 = g + j * G::ST1;
    const float4 Ak = s[pidx<float4>(k2)];
    float4 Mk = s[pidx<float4>((L - k2) & (L - 1))];
    if (k2 == 0) Mk = make_float4(0.f, 0.f, 0.f, 0.f);  // C(., N2) = 0
    const float2 bk = __ldg(a.ib + k2);
    float2 va, vb;
    if (k1a == 0) {
      // V(0,k2) = conj(a_0) conj(b) [C(0,k2) - i C(0,N2-k2)]
      // V(h,k2) = conj(a_h) conj(b) [(C(h,k2) - C(h,N2-k2)) - i (C(h,k2) + C(h,N2-k2))]
      const float2 v0 = cmul(cmul(make_float2(Ak.x, -Mk.x), bk), ia_a);
      const float2 vh = cmul(cmul(make_float2(Ak.y - Mk.y, -(Ak.y + Mk.y)), bk), ia_h);
      va = make_float2(v0.x - vh.y, v0.y + vh.x);  // V(0) + i V(h)
    } else {
      va = cmul(cmul(make_float2(Ak.x - Mk.y, -(Ak.y + Mk.x)), bk), ia_a);
    }
    vb = cmul(cmul(make_float2(Ak.z - Mk.w, -(Ak.w + Mk.z)), bk), ia_b);
    v[j] = pack2(va, vb);
  }
  __syncthreads();  // every staged column consumed before the FFT reuses the buffer
  first_stage_regs<L, true>(v, s, g);
  __syncthreads();
  if constexpr (G::R1 == L) {
    if (valid)
      for (int i = g; i < L; i += G::TPS) Wp[(long long)m * L + i] = s[pidx<float4>(i)];
  } else {
    fft_stages_last_regs<L, G::R1, true>(s, g, a.tw2, v);
    constexpr int NL = last_stage_ns(L);
    constexpr int RL = stage_radix(L, NL);
    constexpr int NB = fft_points(L) / RL;
    if (valid) {
#pragma unroll
      for (int qb = 0; qb < NB; ++qb)
#pragma unroll
        for (int mm = 0; mm < RL; ++mm)
          Wp[(long long)m * L + stage_out_index<L, NL>(g + qb * G::TPS, mm)] = v[qb * RL + mm];
    }
  }
}

// ----------------------------------------------------------------------------
// Inverse, column pass: Hermitian rebuild + inverse FFT along k1 + un-reorder
// ----------------------------------------------------------------------------
// Pair q = complex columns (2q, 2q+1).  Column p of the workspace holds
// U(k1, p) for k1 < N1/2 (row 0: U(0,p) + i U(N1/2,p)), and U(N1-k1, p) =
// conj U(k1, p).  Two real columns p and N2-1-p are rebuilt as one complex
// column Z = U(., p) + i U(., N2-1-p); its inverse FFT is v(., p) + i v(., N2-1-p),
// stored at input columns (2p, 2p+1) of rows s1(n1) (Eq. 2d_idct_post).
template <int L>
__global__ void __launch_bounds__(PairGeom<L>::THREADS, PairGeom<L>::MINB)
k_inv_cols2(Dct2dArgs a) {
  using G = PairGeom<L>;
  extern __shared__ float4 sm4[];
  const int tid = threadIdx.x;
  const int lp = tid / G::TPS, g = tid % G::TPS;
  const int N2 = a.n2;
  const int npairs = N2 >> 2;
  int q = blockIdx.x * G::PB + lp;
  const bool valid = q < npairs;
  if (!valid) q = npairs - 1;
  float4* s = sm4 + lp * G::LP;
  const float4* Wp = reinterpret_cast<const float4*>(a.work + (long long)blockIdx.y * a.work_bstride);
  float* x = a.out + (long long)blockIdx.y * a.out_bstride;

  for (int kk = g; kk < L / 4; kk += G::TPS) {
    const int k = 2 * kk;
    const float4* row = Wp + (long long)kk * N2;
    const float4 P0 = row[2 * q];           // W(k, 2q),   W(k+1, 2q)
    const float4 P1 = row[2 * q + 1];       // W(k, 2q+1), W(k+1, 2q+1)
    const float4 Q0 = row[N2 - 1 - 2 * q];  // W(k, N2-1-2q), W(k+1, ...)  (mirror of 2q)
    const float4 Q1 = row[N2 - 2 - 2 * q];  // mirror of 2q+1
    // Z_h(kr) for h = 0, 1 and kr = k, k+1 (plus the conjugate-side entries)
    float2 zk[2], zm[2], zk1[2], zm1[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4 Pw = h ? P1 : P0, Qw = h ? Q1 : Q0;
      const float2 wp = lo(Pw), wq = lo(Qw), wp1 = hi(Pw), wq1 = hi(Qw);
      if (k == 0) {
        zk[h] = make_float2(wp.x, wq.x);   // Z(0)
        zm[h] = make_float2(wp.y, wq.y);   // Z(L/2)
      } else {
        zk[h] = make_float2(wp.x - wq.y, wp.y + wq.x);  // Z(k)
        zm[h] = make_float2(wp.x + wq.y, wq.x - wp.y);  // Z(L-k)
      }
      zk1[h] = make_float2(wp1.x - wq1.y, wp1.y + wq1.x);
      zm1[h] = make_float2(wp1.x + wq1.y, wq1.x - wp1.y);
    }
    s[pidx<float4>(k)] = pack2(zk[0], zk[1]);
    s[pidx<float4>(k == 0 ? L / 2 : L - k)] = pack2(zm[0], zm[1]);
    s[pidx<float4>(k + 1)] = pack2(zk1[0], zk1[1]);
    s[pidx<float4>(L - k - 1)] = pack2(zm1[0], zm1[1]);
  }
  __syncthreads();
  float4 v[fft_points(L)];
  fft_stages_last_regs<L, 1, true>(s, g, a.tw1, v);
  constexpr int NL = last_stage_ns(L);
  constexpr int RL = stage_radix(L, NL);
  constexpr int NB = fft_points(L) / RL;
  if (valid) {
#pragma unroll
    for (int qb = 0; qb < NB; ++qb)
#pragma unroll
      for (int mm = 0; mm < RL; ++mm) {
        const int n = stage_out_index<L, NL>(g + qb * G::TPS, mm);
        *(reinterpret_cast<float4*>(x + (long long)reorder_src(n, L) * N2) + q) = v[qb * RL + mm];
      }
  }
}

}  // namespace gbdct
