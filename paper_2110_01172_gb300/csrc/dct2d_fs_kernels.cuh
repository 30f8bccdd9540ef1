// dct2d_fs_kernels.cuh - 2D DCT-II / inverse with four-step column FFTs.
//
// Method: arXiv 2110.01172, Algorithm 2 with the fused pre/postprocess of
// Section III.  The column FFT (length N1 = A*B) is split the four-step way
// so that every global access is a contiguous row segment:
//
//   n1 = n1a + A n1b,   k1 = k1b + B k1a,
//   Z(k1) = sum_n1a W_A^{n1a k1a} [ W_N1^{n1a k1b} sum_n1b z(n1a + A n1b) W_B^{n1b k1b} ].
//
//  * step C1 (per n1a, per block of 128 complex columns): loads the B input
//    rows n1a + A n1b (the reorder of Eq. 2d_dct_pre picks which input rows),
//    a DFT_B per column in registers, the W_N1 twiddle, and stores row
//    k1b*A + n1a of the workspace;
//  * step C2 (per k1b): loads the A workspace rows k1b*A + n1a, a DFT_A per
//    column, and stores Z(k1b + B k1a) in place at row k1b*A + k1a;
//  * the row pass reads rows k1 and N1-k1 of Z, splits the two real columns
//    packed in each complex column, runs the row FFT on the radix-64 engine
//    and writes the symmetric-pair postprocess (Eqs. four-elements, s-t).
//
// The inverse runs the mirror image: the row pass does the four-read
// preprocess (Eq. 2d_idct_pre) and the row IFFT, then pairs columns p and
// N2-1-p into Z(k1) = U(k1,p) + i U(k1,N2-1-p) for k1 and N1-k1 (Hermitian
// rebuild); steps C2' and C1' run the inverse column FFT and C1' stores the
// real column pair with the inverse reorder of Eq. 2d_idct_post.
//
// Workspace: N1 rows of N2/2 complex (row k1 of Z at physical row
// (k1 % B) * A + k1 / B).  Supported: N1 in {1024, 2048, 4096}, N2 in
// {4096, 8192}.
#pragma once

#include "dct2d_r64_kernels.cuh"

namespace gbdct {

constexpr int kFsCols = 128;  // complex columns per column-step CTA (one per thread)

template <int N1>
struct FsGeom {
  static constexpr int A = (N1 == 1024) ? 32 : 64;
  static constexpr int B = N1 / A;
  static constexpr int ROWS = A > B ? A : B;
  static constexpr size_t SMEM = (size_t)ROWS * kFsCols * sizeof(float2);
};

template <int N1>
__device__ __forceinline__ int fs_prow(int k1) {
  return (k1 % FsGeom<N1>::B) * FsGeom<N1>::A + k1 / FsGeom<N1>::B;
}

// Coalesced copy of NR row segments of 128 complex (1 KB) between global
// memory and the [NR][128] float2 staging buffer; `row(i)` gives the global
// float4 pointer of segment i.
template <int NR, bool TO_SMEM, typename RowFn>
__device__ __forceinline__ void fs_copy_rows(float4* stage, RowFn row) {
  constexpr int Q = kFsCols / 2;  // float4 per segment
#pragma unroll 4
  for (int i = threadIdx.x; i < NR * Q; i += kFsCols) {
    const int r = i / Q, q = i % Q;
    if constexpr (TO_SMEM) stage[i] = __ldg(row(r) + q);
    else row(r)[q] = stage[i];
  }
}

// ----------------------------------------------------------------------------
// Forward step C1: reordered input rows -> DFT_B -> twiddle -> workspace
// ----------------------------------------------------------------------------
template <int N1>
__global__ void __launch_bounds__(kFsCols, 3)
k_fs_fwd_c1(Dct2dArgs a, const float2* __restrict__ fstw) {
  using G = FsGeom<N1>;
  extern __shared__ float4 sfs[];
  float2* st = reinterpret_cast<float2*>(sfs);
  const int n1a = blockIdx.x, cb = blockIdx.y;
  const int N2 = a.n2;
  const float4* x4 = reinterpret_cast<const float4*>(a.in + (long long)blockIdx.z * a.in_bstride);
  float4* Z4 = reinterpret_cast<float4*>(a.work + (long long)blockIdx.z * a.work_bstride);
  const int c = threadIdx.x;

  fs_copy_rows<G::B, true>(sfs, [&](int n1b) {
    return x4 + (long long)reorder_src(n1a + G::A * n1b, N1) * (N2 / 4) + cb * (kFsCols / 2);
  });
  __syncthreads();
  float2 v[G::B];
#pragma unroll
  for (int j = 0; j < G::B; ++j) v[j] = st[j * kFsCols + c];
  r64::dft<G::B, false>(v);
#pragma unroll
  for (int k = 1; k < G::B; ++k) v[k] = cmul(v[k], __ldg(fstw + n1a * G::B + k));
  __syncthreads();
#pragma unroll
  for (int k = 0; k < G::B; ++k) st[k * kFsCols + c] = v[k];
  __syncthreads();
  fs_copy_rows<G::B, false>(sfs, [&](int k1b) {
    return Z4 + (long long)(k1b * G::A + n1a) * (N2 / 4) + cb * (kFsCols / 2);
  });
}

// ----------------------------------------------------------------------------
// Forward step C2 / inverse step C2': DFT_A along n1a, in place
// ----------------------------------------------------------------------------
// Forward: rows k1b*A + n1a hold Y(n1a, k1b); writes Z(k1b + B k1a) to rows
// k1b*A + k1a.  Inverse: rows k1b*A + k1a hold Z(k1b + B k1a); writes
// conj(W_N1^{n1a k1b}) sum_k1a Z W_A^{-n1a k1a} to rows k1b*A + n1a.
template <int N1, bool INV>
__global__ void __launch_bounds__(kFsCols, 3)
k_fs_c2(Dct2dArgs a, const float2* __restrict__ fstw) {
  using G = FsGeom<N1>;
  extern __shared__ float4 sfs[];
  float2* st = reinterpret_cast<float2*>(sfs);
  const int k1b = blockIdx.x, cb = blockIdx.y;
  const int N2 = a.n2;
  float4* Z4 = reinterpret_cast<float4*>(a.work + (long long)blockIdx.z * a.work_bstride);
  const int c = threadIdx.x;
  auto rowp = [&](int i) { return Z4 + (long long)(k1b * G::A + i) * (N2 / 4) + cb * (kFsCols / 2); };

  fs_copy_rows<G::A, true>(sfs, rowp);
  __syncthreads();
  float2 v[G::A];
#pragma unroll
  for (int j = 0; j < G::A; ++j) v[j] = st[j * kFsCols + c];
  r64::dft<G::A, INV>(v);
  if (INV) {
#pragma unroll
    for (int n = 1; n < G::A; ++n) v[n] = cmulc(v[n], __ldg(fstw + n * G::B + k1b));
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < G::A; ++k) st[k * kFsCols + c] = v[k];
  __syncthreads();
  fs_copy_rows<G::A, false>(sfs, rowp);
}

// ----------------------------------------------------------------------------
// Inverse step C1': DFT_B along k1b -> inverse reorder into the output rows
// ----------------------------------------------------------------------------
template <int N1>
__global__ void __launch_bounds__(kFsCols, 3)
k_fs_inv_c1(Dct2dArgs a) {
  using G = FsGeom<N1>;
  extern __shared__ float4 sfs[];
  float2* st = reinterpret_cast<float2*>(sfs);
  const int n1a = blockIdx.x, cb = blockIdx.y;
  const int N2 = a.n2;
  const float4* Z4 = reinterpret_cast<const float4*>(a.work + (long long)blockIdx.z * a.work_bstride);
  float4* x4 = reinterpret_cast<float4*>(a.out + (long long)blockIdx.z * a.out_bstride);
  const int c = threadIdx.x;

  fs_copy_rows<G::B, true>(sfs, [&](int k1b) {
    return Z4 + (long long)(k1b * G::A + n1a) * (N2 / 4) + cb * (kFsCols / 2);
  });
  __syncthreads();
  float2 v[G::B];
#pragma unroll
  for (int j = 0; j < G::B; ++j) v[j] = st[j * kFsCols + c];
  r64::dft<G::B, true>(v);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < G::B; ++k) st[k * kFsCols + c] = v[k];
  __syncthreads();
  fs_copy_rows<G::B, false>(sfs, [&](int n1b) {
    return x4 + (long long)reorder_src(n1a + G::A * n1b, N1) * (N2 / 4) + cb * (kFsCols / 2);
  });
}

// ----------------------------------------------------------------------------
// Forward row pass (L = N2): split in the loads, row FFT, postprocess
// ----------------------------------------------------------------------------
// CTA b handles k1 = 2b + s.  Row k1 >= 1 gives output rows k1 and N1-k1; the
// pair (0, N1/2) is one packed sequence V1(0,.) + i V1(N1/2,.).
template <int N1, int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_fs_fwd_rows(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int k1 = 2 * blockIdx.x + s;
  const bool packed = (k1 == 0);
  const int kmir = packed ? N1 / 2 : N1 - k1;
  const float2* Zw = a.work + (long long)blockIdx.z * a.work_bstride;
  const float2* za_row = Zw + (long long)fs_prow<N1>(k1) * (L / 2);
  const float2* zb_row = Zw + (long long)fs_prow<N1>(kmir) * (L / 2);
  float* y = a.out + (long long)blockIdx.z * a.out_bstride;

  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int n2 = t + j * G::ST1;
    const bool lowhalf = n2 < L / 2;
    const int p = lowhalf ? n2 : L - 1 - n2;
    const float2 za = za_row[p];
    const float2 zb = zb_row[p];
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
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) buf[r64::pidx(r64::out_pos<L>(t, qb, m))] = v[qb * G::RL + m];
  __syncthreads();

  const float2 av = __ldg(a.fa + k1);
  float* row0 = y + (long long)k1 * L;
  float* row1 = y + (long long)kmir * L;
  constexpr float RH = 0.70710678118654752f;
  for (int i = t; i < L / 8; i += G::TPS) {
    const int c = 4 * i;
    float2 Yq[5], Ym[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      Yq[d] = buf[r64::pidx(c + d)];
      Ym[d] = buf[r64::pidx((L - c - d) & (L - 1))];
    }
    float q0[4], q1[4], r0[4], r1[4];
#pragma unroll
    for (int d = 1; d <= 3; ++d) {
      const float2 bt = __ldg(a.fb + c + d);
      const float2 P = Yq[d], M = Ym[d];
      if (packed) {
        const float2 s0 = cmul(bt, make_float2(P.x + M.x, P.y - M.y));
        const float2 sh = cmul(bt, make_float2(RH * (P.y + M.y), RH * (M.x - P.x)));
        q0[d] = s0.x;
        q1[d] = sh.x;
        r0[4 - d] = -s0.y;
        r1[4 - d] = -sh.y;
      } else {
        const float2 aP = cmul(P, av);
        const float2 aM = cmul(M, av);
        const float2 sv = cmul(bt, make_float2(aP.x + aM.x, aP.y - aM.y));
        const float2 tv = cmul(bt, make_float2(aP.x - aM.x, aP.y + aM.y));
        q0[d] = sv.x;
        q1[d] = -tv.y;
        r0[4 - d] = -sv.y;
        r1[4 - d] = -tv.x;
      }
    }
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
// Inverse row pass (L = N2): four-read preprocess + row IFFT + column pairing
// ----------------------------------------------------------------------------
template <int N1, int L>
__global__ void __launch_bounds__(R64Geom<L>::THREADS)
k_fs_inv_rows(Dct2dArgs a) {
  using G = R64Geom<L>;
  extern __shared__ float4 smr[];
  const int s = threadIdx.x & 1, t = threadIdx.x >> 1;
  float2* buf = reinterpret_cast<float2*>(smr) + s * G::LP;
  const int k1 = 2 * blockIdx.x + s;
  const bool packed = (k1 == 0);
  const int kmir = packed ? N1 / 2 : N1 - k1;
  const float* C = a.in + (long long)blockIdx.z * a.in_bstride;
  const float* ca = C + (long long)k1 * L;
  const float* cb = C + (long long)kmir * L;
  float2* Zw = a.work + (long long)blockIdx.z * a.work_bstride;
  const float2 ia = __ldg(a.ia + k1);
  const float2 ih = __ldg(a.ia + N1 / 2);

  float2 v[r64::PMAX];
#pragma unroll
  for (int j = 0; j < G::R1; ++j) {
    const int k2 = t + j * G::ST1;
    const int km = (L - k2) & (L - 1);
    const float c1 = __ldg(ca + k2), c3 = __ldg(cb + k2);
    const float c4 = k2 ? __ldg(ca + km) : 0.f;
    const float c2 = k2 ? __ldg(cb + km) : 0.f;
    const float2 bk = __ldg(a.ib + k2);
    if (packed) {
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
#pragma unroll
  for (int qb = 0; qb < G::NBL; ++qb)
#pragma unroll
    for (int m = 0; m < G::RL; ++m) buf[r64::pidx(r64::out_pos<L>(t, qb, m))] = v[qb * G::RL + m];
  __syncthreads();

  // Z_p(k1) = U(k1,p) + i U(k1,L-1-p), Z_p(N1-k1) = conj U(k1,p) + i conj U(k1,L-1-p);
  // packed: U(0,.) + i U(N1/2,.) -> Z_p(0) from the real parts, Z_p(N1/2) from the imaginary.
  float2* zr0 = Zw + (long long)fs_prow<N1>(k1) * (L / 2);
  float2* zr1 = Zw + (long long)fs_prow<N1>(kmir) * (L / 2);
  for (int p = t; p < L / 2; p += G::TPS) {
    const float2 u = buf[r64::pidx(p)];
    const float2 w = buf[r64::pidx(L - 1 - p)];
    if (packed) {
      zr0[p] = make_float2(u.x, w.x);
      zr1[p] = make_float2(u.y, w.y);
    } else {
      zr0[p] = make_float2(u.x - w.y, u.y + w.x);
      zr1[p] = make_float2(u.x + w.y, w.x - u.y);
    }
  }
}

}  // namespace gbdct
