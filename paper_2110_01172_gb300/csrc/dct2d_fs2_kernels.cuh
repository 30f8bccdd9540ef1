// dct2d_fs2_kernels.cuh - four-step column FFTs + row passes, occupancy-first.
//
// Same method and data flow as dct2d_fs_kernels.cuh (arXiv 2110.01172,
// Algorithm 2 with the fused pre/postprocess of Section III; the column FFT of
// length N1 = A*B split the four-step way so that every global access is a
// contiguous row segment), with kernels shaped for occupancy:
//
//  * column steps: a CTA owns a slab of S rows (S = A or B) x a block of
//    complex columns; Q threads share a column group and each holds T = S/Q
//    points of it, so a DFT_S is a DFT_T in registers, a twiddle W_S^{q m},
//    an exchange through shared memory and DFT_Qs
//    (W_S^{(q+Qj)(m+Tp)} = W_S^{qm} W_Q^{qp} W_T^{jm}).  The default vector
//    form (k_fs2_colv) gives each thread two adjacent columns (16-byte
//    accesses; Q = 4 or 8, S up to 128); the scalar form (k_fs2_col) one
//    column with Q = 4;
//  * row passes: one sequence per 16-point thread group (float2), the radix-16
//    Stockham engine of fft_core.cuh, ~64 registers per thread.
//
// Workspace layout as in dct2d_fs_kernels.cuh: N1 rows of N2/2 complex, row
// k1 of the column spectrum at physical row (k1 % B) * A + k1 / B.
// Supported: N1 in {256, ..., 8192} (8192 with the vector column steps only),
// N2 in {256, ..., 16384}.
//
// The other kinds are index/sign maps around the DCT-II (Section V-B, Eq.
// idxst; DST-II per axis), folded into the first loads and last stores
// (a.vkind):
//   DST-II forward   x(n1,n2) (-1)^(n1+n2) in C1's loads; output (k1,k2) stored
//                    at (N1-1-k1, N2-1-k2) by the row pass
//   DST-II inverse   input read at (N1-1-k1, N2-1-k2) by the row pass's staging;
//                    (-1)^(n1+n2) in C1''s stores
//   IDCT_IDXST       input column k2 taken from column N2-k2 (column 0 zero):
//                    the preprocess swaps its reads k2 <-> N2-k2; (-1)^n2 in C1'
//   IDXST_IDCT       input row k1 taken from row N1-k1 (row 0 zero): the row
//                    pass swaps its two rows; (-1)^n1 in C1''s stores
#pragma once

#include "dct2d_kernels.cuh"
#include "fft_soa.cuh"
#include "l2_hint.cuh"

#include <type_traits>

namespace gbdct {

// Calls f(integral_constant<int, I>) for I = B .. E-1 (compile-time loop).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// Four-step split N1 = A * B of the column FFT (a tile parameter: the slabs of
// the column steps are A or B rows); both factors in {16, 32, 64, 128}.
template <int N1, int A_>
struct Fs2Geom {
  static constexpr int A = A_;
  static constexpr int B = N1 / A_;
  static_assert(A >= 16 && A <= 128 && B >= 16 && B <= 128, "four-step factors out of range");
};

// Physical workspace row of column-spectrum row k1 (A, B powers of two).
__device__ __forceinline__ int fs2_prow(int k1, int A, int B) { return (k1 & (B - 1)) * A + k1 / B; }

// ----------------------------------------------------------------------------
// Column steps, vector form (k_fs2_colv): each thread owns CPT adjacent complex
// columns (CPT = 2: 16-byte loads and stores) and T = S/Q points of each; Q
// threads share a column group.  DFT_S = DFT_T in registers, twiddle
// W_S^{q m}, one exchange through shared memory, then DFT_Q across the Q
// threads (S = Q T: W_S^{(q + Q j)(m + T p)} = W_S^{q m} W_Q^{q p} W_T^{j m}).
//   S = 16: Q 4, CPT 2;  S = 32: Q 4, CPT 2;  S = 64: Q 8, CPT 2;
//   S = 128: Q 8, CPT 1 (N1 = 8192).
// ----------------------------------------------------------------------------

// cos(2 pi k / 128), k = 0..127 (float roundings of the exact values)
__host__ __device__ constexpr float cos128(int k) {
  constexpr float t[128] = {
    1.000000000e+00f,
    9.987954562e-01f,
    9.951847267e-01f,
    9.891765100e-01f,
    9.807852804e-01f,
    9.700312532e-01f,
    9.569403357e-01f,
    9.415440652e-01f,
    9.238795325e-01f,
    9.039892931e-01f,
    8.819212643e-01f,
    8.577286100e-01f,
    8.314696123e-01f,
    8.032075315e-01f,
    7.730104534e-01f,
    7.409511254e-01f,
    7.071067812e-01f,
    6.715589548e-01f,
    6.343932842e-01f,
    5.956993045e-01f,
    5.555702330e-01f,
    5.141027442e-01f,
    4.713967368e-01f,
    4.275550934e-01f,
    3.826834324e-01f,
    3.368898534e-01f,
    2.902846773e-01f,
    2.429801799e-01f,
    1.950903220e-01f,
    1.467304745e-01f,
    9.801714033e-02f,
    4.906767433e-02f,
    6.123233996e-17f,
    -4.906767433e-02f,
    -9.801714033e-02f,
    -1.467304745e-01f,
    -1.950903220e-01f,
    -2.429801799e-01f,
    -2.902846773e-01f,
    -3.368898534e-01f,
    -3.826834324e-01f,
    -4.275550934e-01f,
    -4.713967368e-01f,
    -5.141027442e-01f,
    -5.555702330e-01f,
    -5.956993045e-01f,
    -6.343932842e-01f,
    -6.715589548e-01f,
    -7.071067812e-01f,
    -7.409511254e-01f,
    -7.730104534e-01f,
    -8.032075315e-01f,
    -8.314696123e-01f,
    -8.577286100e-01f,
    -8.819212643e-01f,
    -9.039892931e-01f,
    -9.238795325e-01f,
    -9.415440652e-01f,
    -9.569403357e-01f,
    -9.700312532e-01f,
    -9.807852804e-01f,
    -9.891765100e-01f,
    -9.951847267e-01f,
    -9.987954562e-01f,
    -1.000000000e+00f,
    -9.987954562e-01f,
    -9.951847267e-01f,
    -9.891765100e-01f,
    -9.807852804e-01f,
    -9.700312532e-01f,
    -9.569403357e-01f,
    -9.415440652e-01f,
    -9.238795325e-01f,
    -9.039892931e-01f,
    -8.819212643e-01f,
    -8.577286100e-01f,
    -8.314696123e-01f,
    -8.032075315e-01f,
    -7.730104534e-01f,
    -7.409511254e-01f,
    -7.071067812e-01f,
    -6.715589548e-01f,
    -6.343932842e-01f,
    -5.956993045e-01f,
    -5.555702330e-01f,
    -5.141027442e-01f,
    -4.713967368e-01f,
    -4.275550934e-01f,
    -3.826834324e-01f,
    -3.368898534e-01f,
    -2.902846773e-01f,
    -2.429801799e-01f,
    -1.950903220e-01f,
    -1.467304745e-01f,
    -9.801714033e-02f,
    -4.906767433e-02f,
    -1.836970199e-16f,
    4.906767433e-02f,
    9.801714033e-02f,
    1.467304745e-01f,
    1.950903220e-01f,
    2.429801799e-01f,
    2.902846773e-01f,
    3.368898534e-01f,
    3.826834324e-01f,
    4.275550934e-01f,
    4.713967368e-01f,
    5.141027442e-01f,
    5.555702330e-01f,
    5.956993045e-01f,
    6.343932842e-01f,
    6.715589548e-01f,
    7.071067812e-01f,
    7.409511254e-01f,
    7.730104534e-01f,
    8.032075315e-01f,
    8.314696123e-01f,
    8.577286100e-01f,
    8.819212643e-01f,
    9.039892931e-01f,
    9.238795325e-01f,
    9.415440652e-01f,
    9.569403357e-01f,
    9.700312532e-01f,
    9.807852804e-01f,
    9.891765100e-01f,
    9.951847267e-01f,
    9.987954562e-01f

  };
  return t[k & 127];
}

// a * W_R^E for R dividing 128, W_R = exp(-2 pi i / R) (forward) or exp(+2 pi i / R).
template <int R, int E, bool INV, typename T>
__device__ __forceinline__ T mul_w128(T a) {
  constexpr int e = ((E * (128 / R)) % 128 + 128) % 128;
  constexpr float c = cos128(e);
  constexpr float s = cos128((160 - e) % 128);  // sin(2 pi e / 128) = cos(2 pi (32 - e) / 128)
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 32) {
    return mul_mj<INV>(a);
  } else if constexpr (e == 64) {
    return cneg(a);
  } else if constexpr (e == 96) {
    return mul_mj<!INV>(a);
  } else if constexpr (e % 32 == 16) {
    return cmul_diag(a, c, (INV ? s : -s) / c);
  } else {
    return cmulk(a, c, INV ? s : -s);
  }
}

template <int S>
struct ColCfg {
  static constexpr int Q = S >= 64 ? 8 : 4;           // threads per column group
  static constexpr int CPT = S >= 128 ? 1 : 2;        // complex columns per thread
  static constexpr int T = S / Q;                     // points per column per thread
  static constexpr int COLS = S >= 128 ? 64 : 128;    // complex columns per CTA
  static constexpr int NG = COLS / CPT;               // column groups per CTA
  static constexpr int THREADS = NG * Q;
  static constexpr size_t SMEM = (size_t)S * COLS * sizeof(float2);
  using V = typename std::conditional<CPT == 2, float4, float2>::type;
};

// x[m] *= W_S^{q m} (m < T) for the thread's warp-uniform q < Q.
template <int S, int Q, int T, bool INV, typename V>
__device__ __forceinline__ void colv_twiddle(V* x, int q) {
  static_for<1, Q>([&](auto qc) {
    constexpr int qq = decltype(qc)::value;
    if (q == qq) {
      static_for<1, T>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        x[m] = mul_w128<S, qq * m, INV>(x[m]);
      });
    }
  });
}

// DFT_S along the slab rows: on entry x[j] = slab row q + Q j (j < T); on return
// x[i Q + p] = output row (q T/Q + i) + T p  (i < T/Q, p < Q).
template <int S, bool INV, typename V>
__device__ __forceinline__ void colv_dft(V* x, int q, int c, V* ex) {
  using C = ColCfg<S>;
  constexpr int Q = C::Q, T = C::T, NG = C::NG, TQ = T / Q;
  dft<T, INV>(x);
  colv_twiddle<S, Q, T, INV>(x, q);
#pragma unroll
  for (int m = 0; m < T; ++m) ex[(q * T + m) * NG + c] = x[m];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TQ; ++i) {
    const int m = q * TQ + i;
    V y[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) y[p] = ex[(p * T + m) * NG + c];
    dft<Q, INV>(y);
#pragma unroll
    for (int p = 0; p < Q; ++p) x[i * Q + p] = y[p];
  }
  __syncthreads();
}

__device__ __forceinline__ float2 vsign(float2 v, float sr, float sc) { return make_float2(sr * v.x, sc * v.y); }
__device__ __forceinline__ float4 vsign(float4 v, float sr, float sc) {
  return make_float4(sr * v.x, sc * v.y, sr * v.z, sc * v.w);
}

template <int N1, int A, int KIND>
__global__ void __launch_bounds__(ColCfg<(KIND == 0 || KIND == 3) ? N1 / A : A>::THREADS,
                                  1024 / ColCfg<(KIND == 0 || KIND == 3) ? N1 / A : A>::THREADS)
k_fs2_colv(Dct2dArgs a) {
  using G = Fs2Geom<N1, A>;
  constexpr bool INV = KIND >= 2;
  constexpr int S = (KIND == 0 || KIND == 3) ? G::B : G::A;
  using C = ColCfg<S>;
  using V = typename C::V;
  constexpr int T = C::T, Q = C::Q, TQ = T / Q;
  extern __shared__ float4 scv[];
  V* ex = reinterpret_cast<V*>(scv);
  const int c = threadIdx.x % C::NG, q = threadIdx.x / C::NG;
  const int r = blockIdx.x;
  const int N2 = a.n2;
  const long long hv = N2 / 2 / C::CPT;  // V elements per workspace row
  const int colv = blockIdx.y * C::NG + c;  // V index within a row
  V* W = reinterpret_cast<V*>(a.work + (long long)blockIdx.z * a.work_bstride);

  // L2 policies: the streamed input / output evict first, the workspace
  // (read again by the next launch of the transform) evicts last
  const uint64_t pol_stream = l2::evict_first(), pol_keep = l2::evict_last();
  V x[T];
#pragma unroll
  for (int j = 0; j < T; ++j) {
    const int i = q + Q * j;  // slab row of this input
    if constexpr (KIND == 0) {
      const float* xin = a.in + (long long)blockIdx.z * a.in_bstride;
      const int row = reorder_src(r + G::A * i, N1);
      x[j] = l2::ld_once(reinterpret_cast<const V*>(xin + (long long)row * N2) + colv, pol_stream);
      if (a.vkind == 1) {  // DST-II: (-1)^(n1 + n2); real columns alternate in parity
        const float sr = (row & 1) ? -1.f : 1.f;
        x[j] = vsign(x[j], sr, -sr);
      }
    } else if constexpr (KIND == 3) {
      x[j] = l2::ld_once(W + (long long)(i * G::A + r) * hv + colv, pol_stream);  // last use of the workspace
    } else {
      x[j] = l2::ld_once(W + (long long)(r * G::A + i) * hv + colv, pol_keep);
    }
  }
  colv_dft<S, INV>(x, q, c, ex);
#pragma unroll
  for (int i = 0; i < TQ; ++i)
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      const int o = q * TQ + i + T * p;  // k1b (KIND 0), k1a (1), n1a (2), n1b (3)
      V y = x[i * Q + p];
      if constexpr (KIND == 0) {
        y = cmul(y, __ldg(a.fstw + r * G::B + o));
        l2::st(W + (long long)(o * G::A + r) * hv + colv, y, pol_keep);
      } else if constexpr (KIND == 2) {
        y = cmulc(y, __ldg(a.fstw + o * G::B + r));
        l2::st(W + (long long)(r * G::A + o) * hv + colv, y, pol_keep);
      } else if constexpr (KIND == 1) {
        l2::st(W + (long long)(r * G::A + o) * hv + colv, y, pol_keep);
      } else {
        float* xo = a.out + (long long)blockIdx.z * a.out_bstride;
        const int row = reorder_src(r + G::A * o, N1);
        if (a.vkind) {  // output signs: (-1)^(n1+n2) DST-II, (-1)^n2 IDCT_IDXST, (-1)^n1 IDXST_IDCT
          const float sr = (a.vkind != 2 && (row & 1)) ? -1.f : 1.f;
          const float sc = (a.vkind != 3) ? -sr : sr;
          y = vsign(y, sr, sc);
        }
        l2::st(reinterpret_cast<V*>(xo + (long long)row * N2) + colv, y, pol_stream);
      }
    }
}

// ----------------------------------------------------------------------------
// Row passes (L = N2).  Item k1 in [0, N1/2) owns the row pair (k1, N1-k1);
// item 0 the packed pair (0, N1/2).  Forward: Hermitian split of the two
// column-spectrum rows, row FFT, symmetric-pair postprocess (Section III-B,
// Eqs. four-elements, s-t) -> output rows k1 and N1-k1.  Inverse: four-read
// preprocess (Eq. 2d_idct_pre, conjugated twiddle, 1/(N1 N2) in the a-table),
// row IFFT, column pairing Z_p(k1) = U(k1,p) + i U(k1,L-1-p) -> workspace.
// One item group per CTA with the rows staged by the threads (k_fs2_rows);
// used for N2 = 16384, where the two-item form below does not fit.
// ----------------------------------------------------------------------------
template <int L>
struct RowGeom {
  static constexpr int TPS = fft_tps(L);
  static constexpr int NI = (256 / TPS) > 0 ? 256 / TPS : 1;  // items per CTA
  static constexpr int THREADS = NI * TPS;
  static constexpr int LP = pad_len<float2>(L);
  static constexpr size_t SMEM = (size_t)NI * LP * sizeof(float2);
  static constexpr int MINB = 1024 / THREADS;  // caps registers at 64 per thread
};

__device__ __forceinline__ int row_mirror(int k1, int N1) { return k1 ? N1 - k1 : N1 / 2; }

// The two source rows (L floats each) of item k1 of batch entry b.  Forward:
// column-spectrum rows k1 and its mirror in the workspace (four-step physical
// order).  Inverse: input rows with the kind's row map folded in: DST-II reads
// rows N1-1-k1 and N1-1-kmir (columns reversed by inv_pre); IDXST_IDCT takes
// row k1 from row N1-k1, so the two rows trade places and the packed item's
// row 0 is zero (*ra = nullptr).
template <int L, bool INV>
__device__ __forceinline__ void row_sources(const Dct2dArgs& a, int b, int k1, const float** ra, const float** rb) {
  const int N1 = a.n1;
  const int kmir = row_mirror(k1, N1);
  if constexpr (!INV) {
    const float2* Zw = a.work + (long long)b * a.work_bstride;
    *ra = reinterpret_cast<const float*>(Zw + (long long)fs2_prow(k1, a.fsA, a.fsB) * (L / 2));
    *rb = reinterpret_cast<const float*>(Zw + (long long)fs2_prow(kmir, a.fsA, a.fsB) * (L / 2));
  } else {
    const float* C = a.in + (long long)b * a.in_bstride;
    int r0 = k1, r1 = kmir;
    if (a.vkind == 1) {
      r0 = N1 - 1 - k1;
      r1 = N1 - 1 - kmir;
    }
    *ra = C + (long long)r0 * L;
    *rb = C + (long long)r1 * L;
    if (a.vkind == 3) {
      if (k1) {
        const float* t = *ra;
        *ra = *rb;
        *rb = t;
      } else {
        *ra = nullptr;
      }
    }
  }
}

// Copies two rows of L floats (row0 -> sf[0, L), row1 -> sf[L, 2L)) into shared
// memory with 16-byte loads (TPS threads); a null row0 is left unwritten.
template <int L, int TPS>
__device__ __forceinline__ void stage_two_rows(float* sf, const float* row0, const float* row1, int g) {
  const float4* a4 = reinterpret_cast<const float4*>(row0);
  const float4* b4 = reinterpret_cast<const float4*>(row1);
  float4* s4 = reinterpret_cast<float4*>(sf);
  constexpr int Q = L / 4;  // float4 per row
  float4 t[2 * Q / TPS];
#pragma unroll
  for (int j = 0; j < Q / TPS; ++j) {
    if (a4) t[j] = a4[g + j * TPS];
    t[Q / TPS + j] = b4[g + j * TPS];
  }
#pragma unroll
  for (int j = 0; j < Q / TPS; ++j) {
    if (a4) s4[g + j * TPS] = t[j];
    s4[Q + g + j * TPS] = t[Q / TPS + j];
  }
}

// Forward split: st holds rows za (L/2 complex) and zb (L/2 complex); returns
// the thread's 16 points n2 = g + j TPS of the row to transform.
template <int L, int TPS>
__device__ __forceinline__ void fwd_split(const float2* st, bool packed, int g, float2* v) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int n2 = g + j * TPS;
    const bool lowhalf = n2 < L / 2;
    const int p = lowhalf ? n2 : L - 1 - n2;
    const float2 za = st[p];
    const float2 zb = st[L / 2 + p];
    if (packed) {
      v[j] = lowhalf ? make_float2(za.x, zb.x) : make_float2(za.y, zb.y);
    } else {
      v[j] = lowhalf ? make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y))
                     : make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
    }
  }
}

// Forward postprocess from the row spectrum in s (padded layout) to output
// rows k1 and kmir of y (DST-II: rows and columns reversed).
template <int L, int TPS>
__device__ __forceinline__ void fwd_post(const float2* s, const Dct2dArgs& a, float* y, int k1, int kmir,
                                         bool packed, int g) {
  const int N1 = a.n1;
  const float2 av = __ldg(a.fa + k1);
  const bool rev = a.vkind == 1;  // DST-II: output (k1, k2) goes to (N1-1-k1, N2-1-k2)
  float* row0 = y + (long long)(rev ? N1 - 1 - k1 : k1) * L;
  float* row1 = y + (long long)(rev ? N1 - 1 - kmir : kmir) * L;
  constexpr float RH = 0.70710678118654752f;
  for (int i = g; i < L / 8; i += TPS) {
    const int c = 4 * i;
    float2 Yq[5], Ym[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      Yq[d] = s[pidx<float2>(c + d)];
      Ym[d] = s[pidx<float2>((L - c - d) & (L - 1))];
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
      if (e) {
        r0[0] = o0;
        r1[0] = o1;
      } else {
        q0[0] = o0;
        q1[0] = o1;
      }
    }
    if (!rev) {
      *reinterpret_cast<float4*>(row0 + c) = make_float4(q0[0], q0[1], q0[2], q0[3]);
      *reinterpret_cast<float4*>(row1 + c) = make_float4(q1[0], q1[1], q1[2], q1[3]);
      *reinterpret_cast<float4*>(row0 + L - c - 4) = make_float4(r0[0], r0[1], r0[2], r0[3]);
      *reinterpret_cast<float4*>(row1 + L - c - 4) = make_float4(r1[0], r1[1], r1[2], r1[3]);
    } else {
      *reinterpret_cast<float4*>(row0 + L - c - 4) = make_float4(q0[3], q0[2], q0[1], q0[0]);
      *reinterpret_cast<float4*>(row1 + L - c - 4) = make_float4(q1[3], q1[2], q1[1], q1[0]);
      *reinterpret_cast<float4*>(row0 + c) = make_float4(r0[3], r0[2], r0[1], r0[0]);
      *reinterpret_cast<float4*>(row1 + c) = make_float4(r1[3], r1[2], r1[1], r1[0]);
    }
  }
}

// Inverse preprocess: sf holds the two source rows (L floats each, raw);
// zero_a: the first row is zero (IDXST_IDCT, packed item).  DST-II reads the
// columns reversed; IDCT_IDXST swaps the reads at k2 and N2-k2 (column 0 zero).
template <int L, int TPS, bool MAPPED>
__device__ __forceinline__ void inv_pre_loop(const float* sf, const Dct2dArgs& a, float2 ia, float2 ih, bool packed,
                                             bool zero_a, int g, float2* v) {
  const bool rev = MAPPED && a.vkind == 1, swapc = MAPPED && a.vkind == 2;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k2 = g + j * TPS;
    const int km = (L - k2) & (L - 1);
    float c1, c3, c4, c2;
    if constexpr (!MAPPED) {
      c1 = zero_a ? 0.f : sf[k2];
      c3 = sf[L + k2];
      c4 = (k2 && !zero_a) ? sf[km] : 0.f;
      c2 = k2 ? sf[L + km] : 0.f;
    } else {
      const int ka = swapc ? km : k2, kb = swapc ? k2 : km;
      const int pa = rev ? L - 1 - ka : ka, pb = rev ? L - 1 - kb : kb;
      const bool z0 = swapc && !k2;
      c1 = (zero_a || z0) ? 0.f : sf[pa];
      c3 = z0 ? 0.f : sf[L + pa];
      c4 = (k2 && !zero_a) ? sf[pb] : 0.f;
      c2 = k2 ? sf[L + pb] : 0.f;
    }
    const float2 bk = __ldg(a.ib + k2);
    if (packed) {
      const float2 v0 = cmul(cmul(make_float2(c1, -c4), bk), ia);
      const float2 vh = cmul(cmul(make_float2(c3 - c2, -(c3 + c2)), bk), ih);
      v[j] = make_float2(v0.x - vh.y, v0.y + vh.x);
    } else {
      v[j] = cmul(cmul(make_float2(c1 - c2, -(c3 + c4)), bk), ia);
    }
  }
}

// Inverse preprocess: sf holds the two source rows (L floats each, raw);
// zero_a: the first row is zero (IDXST_IDCT, packed item).  DST-II reads the
// columns reversed; IDCT_IDXST swaps the reads at k2 and N2-k2 (column 0 zero).
// The kind is tested once, outside the unrolled loop.
template <int L, int TPS>
__device__ __forceinline__ void inv_pre(const float* sf, const Dct2dArgs& a, int k1, bool packed, bool zero_a,
                                        int g, float2* v) {
  const float2 ia = __ldg(a.ia + k1);
  const float2 ih = __ldg(a.ia + a.n1 / 2);
  if (a.vkind == 1 || a.vkind == 2)
    inv_pre_loop<L, TPS, true>(sf, a, ia, ih, packed, zero_a, g, v);
  else
    inv_pre_loop<L, TPS, false>(sf, a, ia, ih, packed, zero_a, g, v);
}

// Inverse pairing: row IFFT in s -> workspace rows of k1 and kmir.
template <int L, int TPS>
__device__ __forceinline__ void inv_pair(const float2* s, float2* zr0, float2* zr1, bool packed, int g) {
  for (int h = g; h < L / 4; h += TPS) {  // two columns p = 2h, 2h + 1 per 16-byte store
    const int p = 2 * h;
    const float2 u0 = s[pidx<float2>(p)], u1 = s[pidx<float2>(p + 1)];
    const float2 w0 = s[pidx<float2>(L - 1 - p)], w1 = s[pidx<float2>(L - 2 - p)];
    float4 o0, o1;
    if (packed) {
      o0 = make_float4(u0.x, w0.x, u1.x, w1.x);
      o1 = make_float4(u0.y, w0.y, u1.y, w1.y);
    } else {
      o0 = make_float4(u0.x - w0.y, u0.y + w0.x, u1.x - w1.y, u1.y + w1.x);
      o1 = make_float4(u0.x + w0.y, w0.x - u0.y, u1.x + w1.y, w1.x - u1.y);
    }
    *reinterpret_cast<float4*>(zr0 + p) = o0;
    *reinterpret_cast<float4*>(zr1 + p) = o1;
  }
}

// Everything of one item after its rows are in shared memory (st: raw rows;
// s: the item's FFT buffer).  Contains __syncthreads: all threads call it.
template <int L, bool INV>
__device__ __forceinline__ void row_item(const Dct2dArgs& a, int b, int k1, const float* st, float2* s, int g,
                                         bool zero_a) {
  using R = RowGeom<L>;
  const bool packed = (k1 == 0);
  const int kmir = row_mirror(k1, a.n1);
  float2 v[16];
  if constexpr (!INV)
    fwd_split<L, R::TPS>(reinterpret_cast<const float2*>(st), packed, g, v);
  else
    inv_pre<L, R::TPS>(st, a, k1, packed, zero_a, g, v);
  __syncthreads();  // st may alias s: every read of the rows precedes the first stage
  first_stage_regs<L, INV>(v, s, g);
  __syncthreads();
  fft_stages<L, 16, INV>(s, g, a.tw2);
  if constexpr (!INV) {
    fwd_post<L, R::TPS>(s, a, a.out + (long long)b * a.out_bstride, k1, kmir, packed, g);
  } else {
    float2* Zw = a.work + (long long)b * a.work_bstride;
    inv_pair<L, R::TPS>(s, Zw + (long long)fs2_prow(k1, a.fsA, a.fsB) * (L / 2),
                        Zw + (long long)fs2_prow(kmir, a.fsA, a.fsB) * (L / 2), packed, g);
  }
}

template <int L, bool INV>
__global__ void __launch_bounds__(RowGeom<L>::THREADS, RowGeom<L>::MINB) k_fs2_rows(Dct2dArgs a) {
  using R = RowGeom<L>;
  extern __shared__ float4 srw[];
  const int li = threadIdx.x / R::TPS, g = threadIdx.x % R::TPS;
  float2* s = reinterpret_cast<float2*>(srw) + li * R::LP;
  const int k1 = blockIdx.x * R::NI + li;
  const float *ra, *rb;
  row_sources<L, INV>(a, blockIdx.z, k1, &ra, &rb);
  stage_two_rows<L, R::TPS>(reinterpret_cast<float*>(s), ra, rb, g);  // raw rows in the FFT buffer
  __syncthreads();
  row_item<L, INV>(a, blockIdx.z, k1, reinterpret_cast<const float*>(s), s, g, ra == nullptr);
}


// ----------------------------------------------------------------------------
// Row passes, two-item form (N2 <= 8192, the default).  A thread group of
// L/16 threads transforms two row items at once in packed two-lane FP32
// arithmetic (fft_soa.cuh): lane a is item k1, lane b item k1 + 1.  The
// forward Hermitian split is fused into the loads (each thread reads its 16
// points of the four column-spectrum rows straight from the workspace, no
// staging copy), and the split's factor 1/2 is folded into the a-twiddle of
// the combine.  The inverse reads its four-read preprocess inputs straight
// from the input rows.  Item 0 (the packed rows 0 and N1/2) takes the
// packed formulas in lane a of the first group.
// ----------------------------------------------------------------------------
template <int L>
struct RowX2Geom {
  static constexpr int TPS = fft_tps(L);                          // threads per item pair
  static constexpr int NP = (256 / TPS) > 0 ? 256 / TPS : 1;      // item pairs per CTA
  static constexpr int THREADS = NP * TPS;
  static constexpr int LP = L + L / 16;                           // padded float4 per item pair
  static constexpr size_t SMEM = (size_t)NP * LP * sizeof(float4);
  // CTAs per SM: two (up to 128 registers) measured faster than three at 80
  // registers, where the compiler serialises the loads of the split
  static constexpr int MINB = THREADS >= 512 ? 1 : 2;
  static constexpr int MINB_INV = THREADS >= 512 ? 1 : 2;
};

// Column-spectrum rows of item k (row k1 and its mirror) in the workspace.
template <int L>
__device__ __forceinline__ void fwd_rows_of(const Dct2dArgs& a, const float2* Zw, int k, const float2** z,
                                            const float2** m) {
  *z = Zw + (long long)fs2_prow(k, a.fsA, a.fsB) * (L / 2);
  *m = Zw + (long long)fs2_prow(row_mirror(k, a.n1), a.fsA, a.fsB) * (L / 2);
}

// First-stage butterfly of thread g of a group of TPS threads, arranged so that
// the butterfly t and its mirror TPS-1-t sit in lanes l and l^m of one warp
// (m = 16, or 15 when a warp holds two 16-thread groups).
template <int TPS>
__device__ __forceinline__ int mirror_lane_butterfly(int g) {
  if constexpr (TPS >= 32) {
    const int w = g >> 5, l = g & 31;
    return l < 16 ? 16 * w + l : TPS + 15 - 16 * w - l;
  } else {
    return g;
  }
}
template <int TPS>
constexpr int mirror_lane_mask() { return TPS >= 32 ? 16 : TPS - 1; }

// Forward split of two items from the workspace into SoA registers: point
// n2 = t + TPS j of u = V_col(k1, :) is (z(p) + conj m(p)) / 2 for n2 < L/2
// (p = n2) and (z(p) - conj m(p)) / 2i above (p = L-1-n2); the 1/2 is left out
// here.  Packed lane a (item 0): u = V_col(0, :) + i V_col(N1/2, :).  Each
// workspace value is read once: the thread reads its low-half points, forms
// both the low value and the high value it implies (for point L-1-n2, which
// belongs to the mirror butterfly TPS-1-t at j' = 15 - j), and the two mirror
// lanes swap the high values.
// Split of point p for both lanes from the column-spectrum values A = z_a(p),
// Am = m_a(p), B = z_b(p), Bm = m_b(p): the low value (point p) into lo, the
// high value (point L-1-p) exchanged with the mirror lane into hi.
template <int MASK>
__device__ __forceinline__ void split_point(float2 A, float2 Am, float2 B, float2 Bm, bool packed, soa::C2& lo,
                                            soa::C2& hi) {
  const float lra = packed ? A.x : A.x + Am.x, lia = packed ? Am.x : A.y - Am.y;
  const float hra = packed ? A.y : A.y + Am.y, hia = packed ? Am.y : Am.x - A.x;
  lo = soa::C2{make_float2(lra, B.x + Bm.x), make_float2(lia, B.y - Bm.y)};
  const float h0 = hra, h1 = B.y + Bm.y, h2 = hia, h3 = Bm.x - B.x;
  hi = soa::C2{make_float2(__shfl_xor_sync(0xffffffffu, h0, MASK), __shfl_xor_sync(0xffffffffu, h1, MASK)),
               make_float2(__shfl_xor_sync(0xffffffffu, h2, MASK), __shfl_xor_sync(0xffffffffu, h3, MASK))};
}

template <int L>
__device__ __forceinline__ void fwd_split_x2(const float2* __restrict__ za, const float2* __restrict__ ma,
                                             const float2* __restrict__ zb, const float2* __restrict__ mb, int t,
                                             bool packed, soa::C2* v) {
  constexpr int TPS = fft_tps(L);
  constexpr int MASK = mirror_lane_mask<TPS>();
  const uint64_t pol = l2::evict_first();  // last use of the workspace
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + TPS * j;
    const float2 A = l2::ld_once(za + p, pol), Am = l2::ld_once(ma + p, pol), B = l2::ld_once(zb + p, pol),
                 Bm = l2::ld_once(mb + p, pol);
    // low point n2 = p (this thread), high point L-1-p (the mirror lane)
    split_point<MASK>(A, Am, B, Bm, packed, v[j], v[15 - j]);
  }
}

// Forward combine (Section III-B, Eqs. four-elements / s-t) of both items from
// the row spectra Y in s, one column pair (c, L-c) per thread and iteration:
// u = aP + conj(aM), w = aP - conj(aM) (P = Y(c), M = Y(L-c)); with s = b u,
// t = b w (b/2 in the table): y(k1,c) = Re s, y(kmir,c) = -Im t,
// y(k1,L-c) = -Im s, y(kmir,L-c) = -Re t.  Packed lane a: a = 1 for row 0
// and w = sqrt(1/2) (M.x - P.x, -(P.y + M.y)) for row N1/2.
template <int L, int ST = 1>
__device__ __forceinline__ void fwd_post_x2(const float4* __restrict__ s, const Dct2dArgs& a, float* y, int k1,
                                            int kb, bool packed, int g) {
  constexpr int TPS = fft_tps(L);
  constexpr float RH = 0.70710678118654752f;
  const int N1 = a.n1;
  const float2 fa0 = __ldg(a.fa + k1), fa1 = __ldg(a.fa + kb);
  // 1/2 of the split folded into the a-twiddle (not for the packed item)
  const float2 avr = make_float2(packed ? 1.f : 0.5f * fa0.x, 0.5f * fa1.x);
  const float2 avi = make_float2(packed ? 0.f : 0.5f * fa0.y, 0.5f * fa1.y);
  const bool rev = a.vkind == 1;  // DST-II: output (k1, k2) goes to (N1-1-k1, N2-1-k2)
  const int kma = row_mirror(k1, N1), kmb = row_mirror(kb, N1);
  float* ya0 = y + (long long)(rev ? N1 - 1 - k1 : k1) * L;
  float* ya1 = y + (long long)(rev ? N1 - 1 - kma : kma) * L;
  float* yb0 = y + (long long)(rev ? N1 - 1 - kb : kb) * L;
  float* yb1 = y + (long long)(rev ? N1 - 1 - kmb : kmb) * L;
  const uint64_t pol = l2::evict_first();  // the output is streamed out
  // magnitude threshold of Section V-A, Eq. image-compression (0: off)
  const float eps = a.thresh;
  auto st = [&](float* p, float v) { l2::st(p, (eps > 0.f && fabsf(v) < eps) ? 0.f : v, pol); };
  auto column = [&](int c) {
    const soa::C2 P = soa::unpack(s[ST * soa::pidx4(c)]);
    const soa::C2 M = soa::unpack(s[ST * soa::pidx4((L - c) & (L - 1))]);
    const soa::C2 aP = soa::mulw(P, avr, avi), aM = soa::mulw(M, avr, avi);
    const soa::C2 u{soa::add2(aP.re, aM.re), soa::sub2(aP.im, aM.im)};
    soa::C2 w{soa::sub2(aP.re, aM.re), soa::add2(aP.im, aM.im)};
    if (packed) {
      w.re.x = RH * (M.re.x - P.re.x);
      w.im.x = -RH * (P.im.x + M.im.x);
    }
    const float2 bt = __ldg(a.fb + c);
    const soa::C2 sv = soa::mulw(u, soa::bc(bt.x), soa::bc(bt.y));
    const soa::C2 tv = soa::mulw(w, soa::bc(bt.x), soa::bc(bt.y));
    const int c0 = rev ? L - 1 - c : c, c1 = rev ? c - 1 : L - c;  // stored columns of c and L-c
    st(ya0 + c0, sv.re.x);
    st(yb0 + c0, sv.re.y);
    st(ya1 + c0, -tv.im.x);
    st(yb1 + c0, -tv.im.y);
    if (c != 0 && c != L / 2) {
      st(ya0 + c1, -sv.im.x);
      st(yb0 + c1, -sv.im.y);
      st(ya1 + c1, -tv.re.x);
      st(yb1 + c1, -tv.re.y);
    }
  };
#pragma unroll 2
  for (int r = 0; r < L / 2 / TPS; ++r) column(g + TPS * r);
  if (g == 0) column(L / 2);
}

template <int L>
__global__ void __launch_bounds__(RowX2Geom<L>::THREADS, RowX2Geom<L>::MINB) k_fs2_rows_fwd_x2(Dct2dArgs a) {
  using R = RowX2Geom<L>;
  extern __shared__ float4 sxf[];
  const int pi = threadIdx.x / R::TPS, g = threadIdx.x % R::TPS;
  float4* s = sxf + pi * R::LP;
  const int k1 = 2 * (blockIdx.x * R::NP + pi);  // items k1 (lane a), k1 + 1 (lane b)
  const float2* Zw = a.work + (long long)blockIdx.z * a.work_bstride;
  const float2 *za, *ma, *zb, *mb;
  fwd_rows_of<L>(a, Zw, k1, &za, &ma);
  fwd_rows_of<L>(a, Zw, k1 + 1, &zb, &mb);
  soa::C2 v[16];
  const bool packed = (k1 == 0);
  const int t = mirror_lane_butterfly<R::TPS>(g);
  fwd_split_x2<L>(za, ma, zb, mb, t, packed, v);
  soa::first_stage<L, false>(v, s, t);
  __syncthreads();
  soa::stages<L, 16, false>(s, g, a.tw2x);
  fwd_post_x2<L>(s, a, a.out + (long long)blockIdx.z * a.out_bstride, k1, k1 + 1, packed, g);
}

// Inverse four-read preprocess (Eq. 2d_idct_pre, conjugated twiddle, 1/(N1 N2)
// in the a-table) of one item at the thread's points k2 = g + TPS j, as
// (x, ia) pairs: x = (c1 - c2, -(c3 + c4)) b_k2 for a normal item, where
// c1 = C(k1,k2), c3 = C(kmir,k2), c4 = C(k1,N2-k2), c2 = C(kmir,N2-k2) (zero
// past the edge).  The kind's maps are folded into the reads: DST-II reads rows
// N1-1-k and columns reversed; IDCT_IDXST swaps the reads at k2 and N2-k2
// (column 0 zero); IDXST_IDCT swaps the item's two rows (row 0 zero).
struct InvRows {
  const float* ra;  // row of c1 / c4 (null: zero row)
  const float* rb;  // row of c3 / c2
};

__device__ __forceinline__ InvRows inv_rows_of(const Dct2dArgs& a, const float* C, int k, int L) {
  const int N1 = a.n1;
  const int kmir = row_mirror(k, N1);
  int r0 = k, r1 = kmir;
  if (a.vkind == 1) {
    r0 = N1 - 1 - k;
    r1 = N1 - 1 - kmir;
  }
  InvRows r{C + (long long)r0 * L, C + (long long)r1 * L};
  if (a.vkind == 3) {
    if (k) {
      const float* t = r.ra;
      r.ra = r.rb;
      r.rb = t;
    } else {
      r.ra = nullptr;
    }
  }
  return r;
}

// One input value: from global memory with the L2 policy, or (STAGED) from a
// copy of the row already in shared memory.
template <bool STAGED>
__device__ __forceinline__ float inv_ld(const float* p, uint64_t pol) {
  if constexpr (STAGED) {
    return *p;
  } else {
    return l2::ld(p, pol);
  }
}

// The four reads c1, c3, c4, c2 of point k2 of one item.
template <int L, bool MAPPED, bool STAGED = false>
__device__ __forceinline__ float4 inv_reads(const InvRows& r, int k2, bool rev, bool swapc, uint64_t pol) {
  const int km = (L - k2) & (L - 1);
  float c1, c3, c4, c2;
  if constexpr (!MAPPED) {
    c1 = r.ra ? inv_ld<STAGED>(r.ra + k2, pol) : 0.f;
    c3 = inv_ld<STAGED>(r.rb + k2, pol);
    c4 = (k2 && r.ra) ? inv_ld<STAGED>(r.ra + km, pol) : 0.f;
    c2 = k2 ? inv_ld<STAGED>(r.rb + km, pol) : 0.f;
  } else {
    const int ka = swapc ? km : k2, kb = swapc ? k2 : km;
    const int pa = rev ? L - 1 - ka : ka, pb = rev ? L - 1 - kb : kb;
    const bool z0 = swapc && !k2;
    c1 = (!r.ra || z0) ? 0.f : inv_ld<STAGED>(r.ra + pa, pol);
    c3 = z0 ? 0.f : inv_ld<STAGED>(r.rb + pa, pol);
    c4 = (k2 && r.ra) ? inv_ld<STAGED>(r.ra + pb, pol) : 0.f;
    c2 = k2 ? inv_ld<STAGED>(r.rb + pb, pol) : 0.f;
  }
  return make_float4(c1, c3, c4, c2);
}

template <int L, bool MAPPED, bool PACKED, bool STAGED = false>
__device__ __forceinline__ void inv_pre_x2(const Dct2dArgs& a, const InvRows& A, const InvRows& B, int k1, int kb,
                                           int g, soa::C2* v) {
  constexpr int TPS = fft_tps(L);
  const bool rev = MAPPED && a.vkind == 1, swapc = MAPPED && a.vkind == 2;
  const float2 iaA = __ldg(a.ia + k1), iaB = __ldg(a.ia + kb);
  const float2 ih = __ldg(a.ia + a.n1 / 2);
  const float2 iar = make_float2(iaA.x, iaB.x), iai = make_float2(iaA.y, iaB.y);
  const uint64_t pol = l2::evict_first();  // the input is streamed in
  // points j and 15 - j back to back: the value read at N2 - k2 is read again
  // as the k2 point of the mirror thread TPS - g at iteration 15 - j, so the
  // two reads of every input value fall close together and the second hits L1
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) {
    const int j = (jj & 1) ? 15 - (jj >> 1) : (jj >> 1);
    const int k2 = g + TPS * j;
    const float4 ca = inv_reads<L, MAPPED, STAGED>(A, k2, rev, swapc, pol);
    const float4 cb = inv_reads<L, MAPPED, STAGED>(B, k2, rev, swapc, pol);
    const float2 bk = __ldg(a.ib + k2);
    // x = (c1 - c2, -(c3 + c4)), v = x b ia
    const soa::C2 x{make_float2(ca.x - ca.w, cb.x - cb.w), make_float2(-(ca.y + ca.z), -(cb.y + cb.z))};
    v[j] = soa::mulw(soa::mulw(x, soa::bc(bk.x), soa::bc(bk.y)), iar, iai);
    if constexpr (PACKED) {  // lane a: rows 0 and N1/2 packed as re / im of one sequence
      const float2 v0 = cmul(cmul(make_float2(ca.x, -ca.z), bk), iaA);
      const float2 vh = cmul(cmul(make_float2(ca.y - ca.w, -(ca.y + ca.w)), bk), ih);
      v[j].re.x = v0.x - vh.y;
      v[j].im.x = v0.y + vh.x;
    }
  }
}

// Inverse pairing of both items: row IFFT u in s -> workspace rows k1 and its
// mirror: Z(k1, p) = u(p) + i u(L-1-p), Z(kmir, p) = conj(u(p)) + i conj(u(L-1-p)),
// one column p per thread and iteration; packed lane a: the real and imaginary
// parts go to rows 0 and N1/2.
template <int L>
__device__ __forceinline__ void inv_pair_x2(const float4* __restrict__ s, const Dct2dArgs& a, float2* Zw, int k1,
                                            bool packed, int g) {
  constexpr int TPS = fft_tps(L);
  float2* za = Zw + (long long)fs2_prow(k1, a.fsA, a.fsB) * (L / 2);
  float2* ma = Zw + (long long)fs2_prow(row_mirror(k1, a.n1), a.fsA, a.fsB) * (L / 2);
  float2* zb = Zw + (long long)fs2_prow(k1 + 1, a.fsA, a.fsB) * (L / 2);
  float2* mb = Zw + (long long)fs2_prow(row_mirror(k1 + 1, a.n1), a.fsA, a.fsB) * (L / 2);
  const uint64_t pol = l2::evict_last();  // read again by the next column step
#pragma unroll 2
  for (int r = 0; r < L / 2 / TPS; ++r) {
    const int p = g + TPS * r;
    const soa::C2 u = soa::unpack(s[soa::pidx4(p)]), w = soa::unpack(s[soa::pidx4(L - 1 - p)]);
    l2::st(zb + p, make_float2(u.re.y - w.im.y, u.im.y + w.re.y), pol);
    l2::st(mb + p, make_float2(u.re.y + w.im.y, w.re.y - u.im.y), pol);
    l2::st(za + p, packed ? make_float2(u.re.x, w.re.x) : make_float2(u.re.x - w.im.x, u.im.x + w.re.x), pol);
    l2::st(ma + p, packed ? make_float2(u.im.x, w.im.x) : make_float2(u.re.x + w.im.x, w.re.x - u.im.x), pol);
  }
}

// MAPPED: the DST-II / IDCT_IDXST index maps folded into the reads (a separate
// instantiation, so the plain DCT-II inverse carries no code for them).
template <int L, bool MAPPED>
__global__ void __launch_bounds__(RowX2Geom<L>::THREADS, RowX2Geom<L>::MINB_INV) k_fs2_rows_inv_x2(Dct2dArgs a) {
  using R = RowX2Geom<L>;
  extern __shared__ float4 sxi[];
  const int pi = threadIdx.x / R::TPS, g = threadIdx.x % R::TPS;
  float4* s = sxi + pi * R::LP;
  const int k1 = 2 * (blockIdx.x * R::NP + pi);
  const float* C = a.in + (long long)blockIdx.z * a.in_bstride;
  const InvRows A = inv_rows_of(a, C, k1, L), B = inv_rows_of(a, C, k1 + 1, L);
  const bool packed = (k1 == 0);
  soa::C2 v[16];
  if (packed)
    inv_pre_x2<L, MAPPED, true>(a, A, B, k1, k1 + 1, g, v);
  else
    inv_pre_x2<L, MAPPED, false>(a, A, B, k1, k1 + 1, g, v);
  soa::first_stage<L, true>(v, s, g);
  __syncthreads();
  soa::stages<L, 16, true>(s, g, a.tw2x);
  inv_pair_x2<L>(s, a, a.work + (long long)blockIdx.z * a.work_bstride, k1, packed, g);
}

}  // namespace gbdct
