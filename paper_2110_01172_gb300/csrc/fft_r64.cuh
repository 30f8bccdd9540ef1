// fft_r64.cuh - radix-64 register FFT engine (at most two shared-memory
// exchanges for L <= 4096).
//
// Every thread holds 64 complex points (float2) of one sequence; a length-L
// FFT is L = 64^a * r Stockham stages, each a radix-64 (or radix-r) DFT done
// entirely in registers, so a 4096-point FFT needs one exchange through shared
// memory instead of two with 16 points per thread, and each exchange moves
// 64 points per thread.  The 64-point DFT is 8 x 8 (DFT8 = 4 x 2, DFT4 with
// trivial twiddles); constant twiddles W_R^e are exact float roundings of
// cos(2 pi k / 64) selected at compile time.  Stage twiddles use the same table
// layout as fft_core.cuh with pmax = 64.
#pragma once

#include <type_traits>

#include "fft_core.cuh"

namespace gbdct {
namespace r64 {

constexpr int PMAX = 64;

__host__ __device__ constexpr int radix(int L, int ns) { return stage_radix_p(L, ns, PMAX); }
__host__ __device__ constexpr int points(int L) { return L >= PMAX ? PMAX : L; }
__host__ __device__ constexpr int tps(int L) { return L / points(L); }
__host__ __device__ constexpr int tw_offset(int L, int ns) { return tw_offset_p(L, ns, PMAX); }
__host__ __device__ constexpr int tw_size(int L) { return tw_size_p(L, PMAX); }
__host__ __device__ constexpr int last_ns(int L) {
  int n = 1;
  while (n * radix(L, n) < L) n *= radix(L, n);
  return n;
}
// Shared-memory layout: two float2 of padding after every 64 points, so that
// the first stage's per-thread runs of 64 outputs (stored as float4 pairs)
// fall on distinct banks.
__host__ __device__ constexpr int pad_len(int L) { return L + 2 * (L / 64); }
__device__ __forceinline__ int pidx(int i) { return i + ((i >> 6) << 1); }

// cos(2 pi k / 64), k = 0..63
__host__ __device__ constexpr float cos64(int k) {
  constexpr float t[64] = {
    1.000000000e+00f,
    9.951847267e-01f,
    9.807852804e-01f,
    9.569403357e-01f,
    9.238795325e-01f,
    8.819212643e-01f,
    8.314696123e-01f,
    7.730104534e-01f,
    7.071067812e-01f,
    6.343932842e-01f,
    5.555702330e-01f,
    4.713967368e-01f,
    3.826834324e-01f,
    2.902846773e-01f,
    1.950903220e-01f,
    9.801714033e-02f,
    6.123233996e-17f,
    -9.801714033e-02f,
    -1.950903220e-01f,
    -2.902846773e-01f,
    -3.826834324e-01f,
    -4.713967368e-01f,
    -5.555702330e-01f,
    -6.343932842e-01f,
    -7.071067812e-01f,
    -7.730104534e-01f,
    -8.314696123e-01f,
    -8.819212643e-01f,
    -9.238795325e-01f,
    -9.569403357e-01f,
    -9.807852804e-01f,
    -9.951847267e-01f,
    -1.000000000e+00f,
    -9.951847267e-01f,
    -9.807852804e-01f,
    -9.569403357e-01f,
    -9.238795325e-01f,
    -8.819212643e-01f,
    -8.314696123e-01f,
    -7.730104534e-01f,
    -7.071067812e-01f,
    -6.343932842e-01f,
    -5.555702330e-01f,
    -4.713967368e-01f,
    -3.826834324e-01f,
    -2.902846773e-01f,
    -1.950903220e-01f,
    -9.801714033e-02f,
    -1.836970199e-16f,
    9.801714033e-02f,
    1.950903220e-01f,
    2.902846773e-01f,
    3.826834324e-01f,
    4.713967368e-01f,
    5.555702330e-01f,
    6.343932842e-01f,
    7.071067812e-01f,
    7.730104534e-01f,
    8.314696123e-01f,
    8.819212643e-01f,
    9.238795325e-01f,
    9.569403357e-01f,
    9.807852804e-01f,
    9.951847267e-01f
  };
  return t[((k % 64) + 64) % 64];
}

// Barrier used between stages: BAR == 0 is __syncthreads(); BAR > 0 is the
// named barrier BAR over NT threads (a thread group inside a larger CTA).
template <int BAR, int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (BAR == 0) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
  }
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// a * W_R^E, W_R = exp(-2 pi i / R) (forward) or exp(+2 pi i / R) (inverse).
template <int R, int E, bool INV, typename T>
__device__ __forceinline__ T mul_w(T a) {
  constexpr int e = ((E * (64 / R)) % 64 + 64) % 64;
  constexpr float c = cos64(e);
  constexpr float s = cos64(16 - e);  // sin(2 pi e / 64)
  if constexpr (e == 0) {
    return a;
  } else if constexpr (e == 16) {
    return mul_mj<INV>(a);
  } else if constexpr (e == 32) {
    return cneg(a);
  } else if constexpr (e == 48) {
    return mul_mj<!INV>(a);
  } else if constexpr (e % 16 == 8) {
    return cmul_diag(a, c, (INV ? s : -s) / c);
  } else {
    return cmulk(a, c, INV ? s : -s);
  }
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(T* v);

// DFT of size R1*R2: input index j = R2 j1 + j2, output index m = m1 + R1 m2.
template <int R1, int R2, bool INV, typename T>
__device__ __forceinline__ void dft_comp(T* v) {
  constexpr int R = R1 * R2;
  static_for<0, R2>([&](auto j2c) {
    constexpr int j2 = decltype(j2c)::value;
    T u[R1];
    static_for<0, R1>([&](auto j1c) {
      constexpr int j1 = decltype(j1c)::value;
      u[j1] = v[R2 * j1 + j2];
    });
    dft<R1, INV>(u);
    static_for<0, R1>([&](auto m1c) {
      constexpr int m1 = decltype(m1c)::value;
      v[R2 * m1 + j2] = mul_w<R, j2 * m1, INV>(u[m1]);
    });
  });
  T out[R];
  static_for<0, R1>([&](auto m1c) {
    constexpr int m1 = decltype(m1c)::value;
    T u[R2];
    static_for<0, R2>([&](auto j2c) {
      constexpr int j2 = decltype(j2c)::value;
      u[j2] = v[R2 * m1 + j2];
    });
    dft<R2, INV>(u);
    static_for<0, R2>([&](auto m2c) {
      constexpr int m2 = decltype(m2c)::value;
      out[m1 + R1 * m2] = u[m2];
    });
  });
  static_for<0, R>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    v[i] = out[i];
  });
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(T* v) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    const T t0 = v[0];
    v[0] = cadd(t0, v[1]);
    v[1] = csub(t0, v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    dft_comp<4, 2, INV>(v);
  } else if constexpr (R == 16) {
    dft_comp<4, 4, INV>(v);
  } else if constexpr (R == 32) {
    dft_comp<8, 4, INV>(v);
  } else if constexpr (R == 64) {
    dft_comp<8, 8, INV>(v);
  }
}

// Twiddle + DFT of butterfly t of the stage starting at NS, on R registers.
template <int L, int NS, bool INV>
__device__ __forceinline__ void butterfly(float2* v, int t, const float2* __restrict__ tw) {
  constexpr int R = radix(L, NS);
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

// First stage: v holds the points t + j * (L / R1), j < R1, of the natural-
// order input; runs the radix-R1 DFT and stores the outputs at t*R1 + m.
template <int L, bool INV>
__device__ __forceinline__ void first_stage(float2* v, float2* __restrict__ s, int t) {
  constexpr int R = radix(L, 1);
  dft<R, INV>(v);
  if constexpr (R % 2 == 0) {
#pragma unroll
    for (int m = 0; m < R; m += 2)
      *reinterpret_cast<float4*>(s + pidx(t * R + m)) = make_float4(v[m].x, v[m].y, v[m + 1].x, v[m + 1].y);
  } else {
#pragma unroll
    for (int m = 0; m < R; ++m) s[pidx(t * R + m)] = v[m];
  }
}

// Stages NS .. L of the sequence at `s` (the caller has synchronised after the
// previous stage's stores).  Intermediate stages go through shared memory; the
// last stage leaves its outputs in v: butterfly qb (< NB) of thread t holds
// outputs (t + qb*TPS) + m * last_ns(L), m < R_last.
template <int L, int NS, bool INV, int BAR = 0, int NT = 0>
__device__ __forceinline__ void stages_to_regs(float2* __restrict__ s, int t, const float2* __restrict__ tw,
                                               float2* v) {
  constexpr int R = radix(L, NS);
  constexpr int TPS = tps(L);
  constexpr int NB = points(L) / R;
  constexpr int STRIDE = L / R;
#pragma unroll
  for (int qb = 0; qb < NB; ++qb) {
    const int tb = t + qb * TPS;
#pragma unroll
    for (int j = 0; j < R; ++j) v[qb * R + j] = s[pidx(tb + j * STRIDE)];
  }
  if constexpr (NS * R < L) {
    group_sync<BAR, NT>();
#pragma unroll
    for (int qb = 0; qb < NB; ++qb) {
      const int tb = t + qb * TPS;
      butterfly<L, NS, INV>(v + qb * R, tb, tw);
      const int k = tb & (NS - 1);
      const int base = (tb - k) * R + k;
#pragma unroll
      for (int m = 0; m < R; ++m) s[pidx(base + m * NS)] = v[qb * R + m];
    }
    group_sync<BAR, NT>();
    stages_to_regs<L, NS * R, INV, BAR, NT>(s, t, tw, v);
  } else {
#pragma unroll
    for (int qb = 0; qb < NB; ++qb) butterfly<L, NS, INV>(v + qb * R, t + qb * TPS, tw);
  }
}

// Output position of register v[qb * R_last + m] after stages_to_regs.
template <int L>
__device__ __forceinline__ int out_pos(int t, int qb, int m) {
  return t + qb * tps(L) + m * last_ns(L);
}

}  // namespace r64
}  // namespace gbdct
