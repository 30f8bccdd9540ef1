// dct_axis0.cu - the axis-0 pass of the 3D transform (see dct_axis0.cuh).
#include "dct_axis0.cuh"

#include "dct2d_kernels.cuh"
#include "fft_core.cuh"
#include "fft_soa.cuh"
#include "l2_hint.cuh"
#include "launch_dep.cuh"

namespace gbdct {
namespace {

template <int N>
struct AxisGeom {
  static constexpr int TPS = fft_tps(N);      // threads per sequence
  static constexpr int PTS = fft_points(N);   // points per thread
  static constexpr int SP = pad_len<float2>(N) + 1;  // odd sequence stride (float2)
};

// Inverse pre of one row of a column pair: c = (X_a[k], X_b[k]), m = (X_a[N-k],
// X_b[N-k]) (zero for k = 0), w = e^{+i pi k / 2N} / N; returns Va[k] + i Vb[k]
// with Va[k] = w (X_a[k] - i X_a[N-k]) and Vb likewise.
__device__ __forceinline__ float2 axis_pre(float2 c, float2 m, float2 w) {
  const float2 va = cmul(make_float2(c.x, -m.x), w);
  const float2 vb = cmul(make_float2(c.y, -m.y), w);
  return make_float2(va.x - vb.y, va.y + vb.x);
}

template <int N, bool INV>
__global__ void __launch_bounds__(512, 2) k_axis0(AxisArgs a) {
  using G = AxisGeom<N>;
  extern __shared__ float4 sax[];
  float2* sm = reinterpret_cast<float2*>(sax);
  const int P = 1 << a.lgP;
  const int t = threadIdx.x;
  const int p = t & (P - 1), rg = t >> a.lgP;  // load/store mapping: column pair, row group
  const long long col = 2 * ((long long)blockIdx.x * P + p);
  const float* X = a.in + (long long)blockIdx.y * a.bstride;
  float* Y = a.out + (long long)blockIdx.y * a.bstride;
  float2* seq = sm + p * G::SP;

  // rows rg, rg + TPS, ...: a strided pointer, eight loads in flight per thread
  const float* src = X + (long long)rg * a.M + col;
  const long long rstep = (long long)G::TPS * a.M;
  pdl::wait_prior_grid();  // the slices' last launch wrote (or reads) this array
  if constexpr (!INV) {
#pragma unroll 8
    for (int j = 0; j < G::PTS; ++j) {
      seq[pidx<float2>(reorder_dst(rg + j * G::TPS, N))] = *reinterpret_cast<const float2*>(src);
      src += rstep;
    }
    __syncthreads();
    fft_stages<N, 1, false>(sm + (t / G::TPS) * G::SP, t % G::TPS, a.tw);
    pdl::launch_dependents();
#pragma unroll
    for (int j = 0; j < G::PTS; ++j) {
      const int k = rg + j * G::TPS;
      const float2 zk = seq[pidx<float2>(k)];
      const float2 zm = seq[pidx<float2>((N - k) & (N - 1))];
      const float2 w = __ldg(a.w + k);  // e^{-i pi k / 2N} / 2
      // 2 Va = Z[k] + conj Z[N-k];  2 Vb = -i (Z[k] - conj Z[N-k])
      const float va_r = zk.x + zm.x, va_i = zk.y - zm.y;
      const float vb_r = zk.y + zm.y, vb_i = zm.x - zk.x;
      *reinterpret_cast<float2*>(Y + (long long)k * a.M + col) =
          make_float2(w.x * va_r - w.y * va_i, w.x * vb_r - w.y * vb_i);
    }
  } else {
#pragma unroll 8
    for (int j = 0; j < G::PTS; ++j) {
      seq[pidx<float2>(rg + j * G::TPS)] = *reinterpret_cast<const float2*>(src);
      src += rstep;
    }
    __syncthreads();
    // Z[k] = Va[k] + i Vb[k] from rows k and N-k; each thread rebuilds both ends
    // of its mirror pairs (k, N-k), k < N/2, in place (k = 0 also does N/2).
#pragma unroll
    for (int j = 0; j < G::PTS / 2; ++j) {
      const int k = rg + j * G::TPS;
      const int km = k ? N - k : N / 2;
      const float2 c = seq[pidx<float2>(k)];   // (X_a[k], X_b[k])
      const float2 m = seq[pidx<float2>(km)];  // (X_a[N-k], X_b[N-k]); row N/2 when k = 0
      seq[pidx<float2>(k)] = axis_pre(c, k ? m : make_float2(0.f, 0.f), __ldg(a.w + k));
      seq[pidx<float2>(km)] = axis_pre(m, k ? c : m, __ldg(a.w + km));
    }
    __syncthreads();
    fft_stages<N, 1, true>(sm + (t / G::TPS) * G::SP, t % G::TPS, a.tw);
    pdl::launch_dependents();
#pragma unroll
    for (int j = 0; j < G::PTS; ++j) {
      const int n = rg + j * G::TPS;
      *reinterpret_cast<float2*>(Y + (long long)reorder_src(n, N) * a.M + col) = seq[pidx<float2>(n)];
    }
  }
}

// A float4 of a row (two adjacent column pairs (re_a, im_a, re_b, im_b)) as
// one point of a two-lane sequence.
__device__ __forceinline__ soa::C2 pairs_to_soa(float4 q) { return {make_float2(q.x, q.z), make_float2(q.y, q.w)}; }

// Packed form, N >= 64: NP two-lane sequences (float4 = two adjacent column
// pairs of a row) per CTA, TPS = N/16 threads each, 128 threads per CTA.
template <int N>
struct AxisSoaGeom {
  static constexpr int TPS = fft_tps(N);
  static constexpr int NP = (128 / TPS) > 0 ? 128 / TPS : 1;
  static constexpr int THREADS = NP * TPS;
  static constexpr int LP = N + N / 16;
  static constexpr size_t SMEM = (size_t)NP * LP * sizeof(float4);
  static constexpr int MINB = THREADS >= 512 ? 1 : 512 / THREADS;  // up to 128 registers
};

template <int N, bool INV>
__global__ void __launch_bounds__(AxisSoaGeom<N>::THREADS, AxisSoaGeom<N>::MINB) k_axis0_soa(AxisArgs a) {
  using G = AxisSoaGeom<N>;
  constexpr int TPS = G::TPS, NP = G::NP;
  extern __shared__ float4 sas[];
  const int pi = threadIdx.x % NP, g = threadIdx.x / NP;
  const long long hv = a.M / 4;  // float4 per row
  const long long vcol = (long long)blockIdx.x * NP + pi;
  const float4* X = reinterpret_cast<const float4*>(a.in + (long long)blockIdx.y * a.bstride) + vcol;
  float4* Y = reinterpret_cast<float4*>(a.out + (long long)blockIdx.y * a.bstride) + vcol;
  float4* s = sas + pi;
  const uint64_t pol = l2::evict_first();
  soa::C2 v[16];
  pdl::wait_prior_grid();
  if constexpr (!INV) {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = pairs_to_soa(l2::ld_once(X + reorder_src(g + TPS * j, N) * hv, pol));
    soa::first_stage<N, false, NP>(v, s, g);
    __syncthreads();
    soa::stages<N, 16, false, NP>(s, g, a.tw4);
    pdl::launch_dependents();
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const int k = g + TPS * r;
      const soa::C2 zk = soa::unpack(s[NP * soa::pidx4(k)]);
      const soa::C2 zm = soa::unpack(s[NP * soa::pidx4((N - k) & (N - 1))]);
      const float2 w = __ldg(a.w + k);  // e^{-i pi k / 2N} / 2
      // per lane: 2 Va = Z[k] + conj Z[N-k], 2 Vb = -i (Z[k] - conj Z[N-k]); X = Re(w 2V)
      const float2 va_r = soa::add2(zk.re, zm.re), va_i = soa::sub2(zk.im, zm.im);
      const float2 vb_r = soa::add2(zk.im, zm.im), vb_i = soa::sub2(zm.re, zk.re);
      const float2 xa = soa::fma2(va_i, soa::bc(-w.y), soa::mul2(va_r, soa::bc(w.x)));
      const float2 xb = soa::fma2(vb_i, soa::bc(-w.y), soa::mul2(vb_r, soa::bc(w.x)));
      l2::st(Y + (long long)k * hv, make_float4(xa.x, xb.x, xa.y, xb.y), pol);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      v[j] = pairs_to_soa(l2::ld_once(X + (long long)(g + TPS * j) * hv, pol));
      s[NP * soa::pidx4(g + TPS * j)] = soa::pack(v[j]);
    }
    __syncthreads();
    // Z[k] = Va[k] + i Vb[k] from rows k and N-k (row N taken as zero)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = g + TPS * j;
      const soa::C2 c = v[j];
      const soa::C2 m = k ? soa::unpack(s[NP * soa::pidx4(N - k)]) : soa::C2{soa::bc(0.f), soa::bc(0.f)};
      const float2 w = __ldg(a.w + k);  // e^{+i pi k / 2N} / N
      // per lane: Va = w (X_a[k] - i X_a[N-k]), Vb = w (X_b[k] - i X_b[N-k]);
      // lane values: X_a = re, X_b = im of the packed column pair
      const soa::C2 va = soa::mulw(soa::C2{c.re, soa::ng(m.re)}, soa::bc(w.x), soa::bc(w.y));
      const soa::C2 vb = soa::mulw(soa::C2{c.im, soa::ng(m.im)}, soa::bc(w.x), soa::bc(w.y));
      v[j] = soa::C2{soa::sub2(va.re, vb.im), soa::add2(va.im, vb.re)};
    }
    __syncthreads();  // the first stage overwrites the staged rows
    soa::first_stage<N, true, NP>(v, s, g);
    __syncthreads();
    soa::stages<N, 16, true, NP>(s, g, a.tw4);
    pdl::launch_dependents();
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const int n = g + TPS * r;
      l2::st(Y + (long long)reorder_src(n, N) * hv, soa::pack_aos(soa::unpack(s[NP * soa::pidx4(n)])), pol);
    }
  }
}

template <int N>
cudaError_t launch_soa(bool inverse, const AxisArgs& a, int batch, cudaStream_t s, bool prepare) {
  using G = AxisSoaGeom<N>;
  if (prepare) {
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_axis0_soa<N, false>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_axis0_soa<N, true>),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    return e;
  }
  const long long ctas = a.M / 4 / G::NP;
  if (a.M % (4LL * G::NP) || ctas < 1 || ctas > 0x7fffffffLL || batch < 1 || batch > 65535)
    return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ctas, (unsigned)batch);
  if (inverse) return pdl::launch(k_axis0_soa<N, true>, grid, dim3(G::THREADS), G::SMEM, s, a);
  return pdl::launch(k_axis0_soa<N, false>, grid, dim3(G::THREADS), G::SMEM, s, a);
}

template <int N>
cudaError_t launch(bool inverse, const AxisArgs& a, int batch, cudaStream_t s, bool prepare) {
  if constexpr (N >= 64) {
    // the packed form where the strip width divides the columns (always for
    // power-of-two slices of at least 4 x 32 elements)
    if (a.tw4 && a.M % (4LL * AxisSoaGeom<N>::NP) == 0) return launch_soa<N>(inverse, a, batch, s, prepare);
  }
  using G = AxisGeom<N>;
  const int P = 1 << a.lgP;
  const size_t smem = (size_t)P * G::SP * sizeof(float2);
  if (prepare) {
    const int pmax = (8192 / N) < 32 ? 8192 / N : 32;  // largest P axis0_lgP picks
    const int lim = pmax * G::SP * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_axis0<N, false>),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k_axis0<N, true>),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
  }
  const long long ctas = a.M / (2LL * P);
  if (ctas < 1 || ctas > 0x7fffffffLL || batch < 1 || batch > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ctas, (unsigned)batch);
  if (inverse) return pdl::launch(k_axis0<N, true>, grid, dim3(P * G::TPS), smem, s, a);
  return pdl::launch(k_axis0<N, false>, grid, dim3(P * G::TPS), smem, s, a);
}

}  // namespace

size_t axis0_smem_bytes(int lgN, int lgP) {
  const int n = 1 << lgN;
  const int sp = (n < 16 ? n : n + (n >> 3)) + 1;
  return (size_t)(1 << lgP) * sp * sizeof(float2);
}

int axis0_threads(int lgN, int lgP) {
  const int n = 1 << lgN;
  return (1 << lgP) * (n >= 16 ? n / 16 : 1);
}

cudaError_t run_axis0(int lgN, bool inverse, const AxisArgs& a, int batch, cudaStream_t s, bool prepare) {
  switch (lgN) {
    case 1: return launch<2>(inverse, a, batch, s, prepare);
    case 2: return launch<4>(inverse, a, batch, s, prepare);
    case 3: return launch<8>(inverse, a, batch, s, prepare);
    case 4: return launch<16>(inverse, a, batch, s, prepare);
    case 5: return launch<32>(inverse, a, batch, s, prepare);
    case 6: return launch<64>(inverse, a, batch, s, prepare);
    case 7: return launch<128>(inverse, a, batch, s, prepare);
    case 8: return launch<256>(inverse, a, batch, s, prepare);
    case 9: return launch<512>(inverse, a, batch, s, prepare);
    case 10: return launch<1024>(inverse, a, batch, s, prepare);
    case 11: return launch<2048>(inverse, a, batch, s, prepare);
    case 12: return launch<4096>(inverse, a, batch, s, prepare);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbdct
