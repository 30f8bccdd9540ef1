// dct2d_tp_kernels.cuh - two-pass family: each direction of the 2D DCT is two
// launches (a column pass and a row pass), the column FFT of length N1 split
// once by decimation in time.
//
// Method: arXiv 2110.01172, Algorithm 2 (reorder, 2D real FFT, postprocess)
// with the fused pre/postprocess of Section III, as in the four-step family
// (dct2d_fs2_kernels.cuh); only the column FFT is organised differently.  With
// M = N1/2 and v the row-reordered input (Eq. 2d_dct_pre), the column DFT of
// length N1 is (radix-2 decimation in time)
//   V[k] = E[k mod M] + W_N1^k O[k mod M],  E = DFT_M(v[2m]),  O = DFT_M(v[2m+1]).
// The column pass computes E and O: a CTA owns a strip of NP complex column
// pairs (NP * 16 bytes of every row) and all M rows of one parity, so the whole
// half-length column FFT runs in shared memory and only E and O are written.
// The row pass applies the radix-2 step while it loads: item k1 needs rows k1
// and N1-k1 of V, and pairing item k1 with item M-k1 makes the four rows of a
// two-item group come from exactly four workspace rows (w = W_N1^k1):
//   V[k1]    = E[k1]   + w O[k1]          V[M+k1] = E[k1]   - w O[k1]
//   V[N1-k1] = E[M-k1] + conj(w) O[M-k1]  V[M-k1] = E[M-k1] - conj(w) O[M-k1]
// The first group pairs the packed item 0 (rows 0 and M = E[0] +- O[0]) with
// item M/2 (rows M/2 and 3M/2 = E[M/2] +- W_N1^{M/2} O[M/2]).
// The inverse is the mirror image: the inverse row pass ends with
//   E'[k] = V[k] + V[M+k],  O'[k] = W_N1^{-k} (V[k] - V[M+k])   (k < M)
// and the inverse column pass takes IDFT_M of E' and O' to the even and odd
// positions of the reordered sequence, stored with the inverse reorder of
// Eq. (2d_idct_post).
//
// Workspace: N1 rows of N2/2 complex; rows [0, M) hold E (E'), rows [M, N1) O (O').
// Supported: N1 in {128, ..., 8192}, N2 in {128, ..., 8192}.
#pragma once

#include "dct2d_fs2_kernels.cuh"
#include "launch_dep.cuh"
#include "tma_util.cuh"

namespace gbdct {

// ----------------------------------------------------------------------------
// Column pass.  A column pair (two adjacent complex columns, one float4 per
// row) is one two-lane sequence of the SoA engine (fft_soa.cuh); the NP pairs
// of a CTA are interleaved point by point in shared memory and thread
// t = g * NP + pi is rank g of pair pi, so a warp's loads and stores cover
// 32/NP rows x NP*16 contiguous bytes.  NP (the strip width, a tile
// parameter the autotuner can choose) keeps the CTA at 64 to 512 threads
// and its shared memory within one SM.
// ----------------------------------------------------------------------------
template <int M, int NP_>
struct TpColGeom {
  static constexpr int TPS = fft_tps(M);  // threads per column pair
  static constexpr int NP = NP_;          // column pairs per CTA
  static constexpr int THREADS = NP * TPS;
  static constexpr int LP = M + M / 16;   // padded points per pair
  static constexpr size_t SMEM = (size_t)NP * LP * sizeof(float4);
  // CTAs per SM: three at 256 threads (80 registers, a few spilled) measured
  // faster than two at 128 registers (4096^2: 35.5 / 33.3 us vs 37.6 / 37.4),
  // the CTAs' strip loads overlapping the others' FFTs; else 128 registers
  static constexpr int MINB = THREADS == 256 ? 3 : (THREADS <= 512 ? 512 / THREADS : 1);
  static constexpr bool VALID = THREADS >= 64 && THREADS <= 512 && SMEM <= 227 * 1024 - 256;
  // bulk tensor copy form: + 128-byte alignment slack, the mbarrier and a flag
  static constexpr size_t SMEM_TMA = SMEM + 256;
  static constexpr int HALF = M / 2;                    // rows of one reorder residue
  static constexpr int ZB = HALF < 256 ? HALF : 256;    // rows per tensor copy (box height)
};
// Default strip width: 128 threads per CTA, but at least two column pairs
// (32 bytes of every row); measured fastest at every size (4096^2: NP = 2,
// 256 threads, 74 / 76 us vs 87 / 87 us at 512 threads).
__host__ __device__ constexpr int tp_default_np(int M) { return 128 / fft_tps(M) > 2 ? 128 / fft_tps(M) : 2; }

__device__ __forceinline__ soa::C2 aos_to_soa(float4 q) { return {make_float2(q.x, q.z), make_float2(q.y, q.w)}; }
__device__ __forceinline__ float4 soa_to_aos(soa::C2 y) { return make_float4(y.re.x, y.im.x, y.re.y, y.im.y); }

// Forward (INV = false): reorder + E or O (blockIdx.y = parity of the
// reordered row) -> workspace.  Inverse: E' or O' -> IDFT_M -> output rows
// with the inverse reorder.
template <int M, int NP, bool INV>
__global__ void __launch_bounds__(TpColGeom<M, NP>::THREADS, TpColGeom<M, NP>::MINB) k_tp_cols(Dct2dArgs a) {
  using G = TpColGeom<M, NP>;
  constexpr int TPS = G::TPS;
  extern __shared__ float4 stc[];
  const int pi = threadIdx.x % G::NP, g = threadIdx.x / G::NP;
  const int par = blockIdx.y;
  const int vcol = blockIdx.x * G::NP + pi;  // float4 column of the strip
  const int N1 = 2 * M;
  const long long hv = a.n2 / 4;             // float4 per row (input, output and workspace)
  float4* W = reinterpret_cast<float4*>(a.work + (long long)blockIdx.z * a.work_bstride) + (long long)par * M * hv +
              vcol;
  float4* s = stc + pi;
  const uint64_t pol_stream = l2::evict_first();
  pdl::wait_prior_grid();
  soa::C2 v[16];
  if constexpr (!INV) {
    const float4* xin = reinterpret_cast<const float4*>(a.in + (long long)blockIdx.z * a.in_bstride) + vcol;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int row = reorder_src(2 * (g + TPS * j) + par, N1);
      float4 q = l2::ld_once(xin + (long long)row * hv, pol_stream);
      if (a.vkind == 1) {  // DST-II: (-1)^(n1 + n2); real columns alternate in parity
        const float sr = (row & 1) ? -1.f : 1.f;
        q = vsign(q, sr, -sr);
      }
      v[j] = aos_to_soa(q);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = aos_to_soa(l2::ld_once(W + (long long)(g + TPS * j) * hv, pol_stream));
  }
  soa::first_stage<M, INV, G::NP>(v, s, g);
  __syncthreads();
  soa::stages<M, 16, INV, G::NP>(s, g, a.tw1x);
  pdl::launch_dependents();
  if constexpr (!INV) {
    const uint64_t pol_keep = l2::evict_last();  // read again by the row pass
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const int k = g + TPS * r;
      l2::st(W + (long long)k * hv, soa_to_aos(soa::unpack(s[G::NP * soa::pidx4(k)])), pol_keep);
    }
  } else {
    float4* xo = reinterpret_cast<float4*>(a.out + (long long)blockIdx.z * a.out_bstride) + vcol;
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
      const int m = g + TPS * r;
      const int row = reorder_src(2 * m + par, N1);
      float4 y = soa_to_aos(soa::unpack(s[G::NP * soa::pidx4(m)]));
      if (a.vkind) {  // output signs: (-1)^(n1+n2) DST-II, (-1)^n2 IDCT_IDXST, (-1)^n1 IDXST_IDCT
        const float sr = (a.vkind != 2 && (row & 1)) ? -1.f : 1.f;
        const float sc = (a.vkind != 3) ? -sr : sr;
        y = vsign(y, sr, sc);
      }
      l2::st(xo + (long long)row * hv, y, pol_stream);
    }
  }
}

// The same pass with the strip moved by bulk tensor copies (TMA) instead of
// per-thread loads and stores, which at 16 * NP bytes per row would cost the
// LSU one wavefront per row touched.  The reorder makes the M rows of one
// parity two regular row sets: with the input viewed as (x, row % 4, row / 4,
// batch), the first half of the reordered positions (m < M/2) is row 4m + 2par
// (residue 2par, z = m) and the second half is row 2N1 - 4m - 2par - 1
// (residue 3 - 2par, z = M - 1 - m), so each is a run of boxes of ZB rows at
// one residue.  The strip lands dense in shared memory (second half in z
// order), the threads take their points from there, and the last FFT stage
// writes its outputs dense (inverse: second half reversed) and interleaved
// (re_a, im_a, re_b, im_b) for the bulk tensor stores.  mx: 4D map of the input (forward) or output (inverse), box
// {4 NP, 1, ZB, 1}; mw: 3D map of the workspace (x, row, batch), box
// {4 NP, ZB, 1}.  One thread issues the copies and waits on the mbarrier
// (bounded; a wait that gives up records the device error, waits again for
// the copies to land and leaves the strip unwritten).
__device__ __forceinline__ float4* align128(float4* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  return reinterpret_cast<float4*>((a + 127) & ~uintptr_t(127));
}

template <int M, int NP, bool INV>
__global__ void __launch_bounds__(TpColGeom<M, NP>::THREADS, TpColGeom<M, NP>::MINB)
    k_tp_cols_tma(Dct2dArgs a, const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw) {
  using G = TpColGeom<M, NP>;
  constexpr int TPS = G::TPS, HALF = G::HALF, ZB = G::ZB;
  extern __shared__ float4 stt_raw[];
  float4* buf = align128(stt_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + NP * G::LP);
  int* flag = reinterpret_cast<int*>(bar + 1);
  const int pi = threadIdx.x % NP, g = threadIdx.x / NP;
  const int par = blockIdx.y, b = blockIdx.z;
  const int x0 = blockIdx.x * NP * 4;  // first float column of the strip
  if (threadIdx.x == 0) {
    tma::bar_init(bar, 1);
    tma::fence_barrier_init();
  }
  pdl::wait_prior_grid();
  if (threadIdx.x == 0) {
    tma::bar_expect_tx(bar, (uint32_t)(M * NP * sizeof(float4)));
    const uint64_t pol = l2::evict_first();  // input streamed once / last use of the workspace
    if constexpr (!INV) {
      for (int z = 0; z < HALF; z += ZB) {
        tma::load_4d(buf + z * NP, &mx, x0, 2 * par, z, b, bar, pol);
        tma::load_4d(buf + (HALF + z) * NP, &mx, x0, 3 - 2 * par, z, b, bar, pol);
      }
    } else {
      for (int z = 0; z < M; z += ZB) tma::load_3d(buf + z * NP, &mw, x0, par * M + z, b, bar, pol);
    }
    const uint32_t polls = a.polls ? a.polls : tma::kDefaultPolls;
    int ok = tma::bar_wait_from_issue(bar, 0, polls);
    if (!ok) {
      atomicExch(a.err, 1);
      tma::bar_wait(bar, 0, tma::kDefaultPolls);  // the copies must land before the CTA exits
    }
    *flag = ok;
  }
  __syncthreads();
  if (!*flag) return;
  // every thread observes the completed phase (acquire of the copied data);
  // it has completed, so the first, non-blocking poll succeeds
  if (threadIdx.x) tma::test_wait(bar, 0);
  soa::C2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int m = g + TPS * j;
    if constexpr (!INV) {
      float4 q = buf[NP * (m < HALF ? m : 3 * HALF - 1 - m) + pi];
      if (a.vkind == 1) {  // DST-II: (-1)^(n1 + n2); rows of the first half even, second half odd
        const float sr = m < HALF ? 1.f : -1.f;
        q = vsign(q, sr, -sr);
      }
      v[j] = aos_to_soa(q);
    } else {
      v[j] = aos_to_soa(buf[NP * m + pi]);
    }
  }
  __syncthreads();
  float4* s = buf + pi;
  soa::first_stage<M, INV, NP>(v, s, g);
  __syncthreads();
  soa::stages<M, 16, INV, NP, INV ? 2 : 1>(s, g, a.tw1x);
  if constexpr (INV) {
    if (a.vkind) {  // output signs: (-1)^(n1+n2) DST-II, (-1)^n2 IDCT_IDXST, (-1)^n1 IDXST_IDCT
#pragma unroll 4
      for (int r = 0; r < 16; ++r) {
        const int pos = g + TPS * r;  // slots of the second half hold odd rows
        const float sr = (a.vkind != 2 && pos >= HALF) ? -1.f : 1.f;
        const float sc = (a.vkind != 3) ? -sr : sr;
        buf[NP * pos + pi] = vsign(buf[NP * pos + pi], sr, sc);
      }
    }
  }
  tma::fence_proxy_async();
  __syncthreads();
  pdl::launch_dependents();
  if (threadIdx.x == 0) {
    if constexpr (!INV) {
      const uint64_t pol = l2::evict_last();  // read again by the row pass
      for (int z = 0; z < M; z += ZB) tma::store_3d(&mw, buf + z * NP, x0, par * M + z, b, pol);
    } else {
      const uint64_t pol = l2::evict_first();
      for (int z = 0; z < HALF; z += ZB) {
        tma::store_4d(&mx, buf + z * NP, x0, 2 * par, z, b, pol);
        tma::store_4d(&mx, buf + (HALF + z) * NP, x0, 3 - 2 * par, z, b, pol);
      }
    }
    tma::commit_group();
    tma::wait_group_read();
  }
}

// ----------------------------------------------------------------------------
// Row passes (L = N2), two items per thread group as in the four-step family:
// group c pairs item c (lane a; the packed item 0 when c = 0) with item
// M - c (lane b; item M/2 when c = 0).
// ----------------------------------------------------------------------------
__device__ __forceinline__ int tp_item_b(int c, int M) { return c ? M - c : M / 2; }

// Row-pass geometry: NP item pairs per CTA, TPS = L/16 threads each.  Wide
// CTAs have 256 threads (the four-step family's row geometry); narrow ones 64,
// for grids that would otherwise leave SMs idle (a single transform with few
// rows: 1024^2 has 256 item pairs, 64 wide CTAs for 152 SMs).  SMEM_STAGED
// adds one 8-byte barrier per group and the CTA's 4-byte flag (16 bytes of
// slack) for the inverse pass's staged rows.  (Staging the forward row pass's
// workspace rows the same way measured slower, 36.2 vs 33.5 us at 4096^2: its
// loads already hit L2 and are read once.)
template <int L, bool NARROW>
struct TpRows {
  static constexpr int TPS = fft_tps(L);
  static constexpr int NP = ((NARROW ? 64 : 256) / TPS) > 0 ? (NARROW ? 64 : 256) / TPS : 1;
  static constexpr int THREADS = NP * TPS;
  static constexpr int LP = L + L / 16;
  static constexpr size_t SMEM = (size_t)NP * LP * sizeof(float4);
  static constexpr size_t SMEM_STAGED = SMEM + (size_t)NP * 8 + 16;
  static constexpr int MINB = THREADS >= 512 ? 1 : 512 / THREADS;  // up to 128 registers
};

template <int L, bool NARROW>
__global__ void __launch_bounds__(TpRows<L, NARROW>::THREADS, TpRows<L, NARROW>::MINB) k_tp_rows_fwd(Dct2dArgs a) {
  using R = TpRows<L, NARROW>;
  constexpr int TPS = R::TPS;
  constexpr int MASK = mirror_lane_mask<TPS>();
  extern __shared__ float4 sxt[];
  const int pi = threadIdx.x / TPS, g = threadIdx.x % TPS;
  float4* s = sxt + pi * R::LP;
  const int M = a.n1 / 2;
  const int c = blockIdx.x * R::NP + pi;
  const bool first = (c == 0);
  const int kb = tp_item_b(c, M);
  const float2* Zw = a.work + (long long)blockIdx.z * a.work_bstride;
  const float2* e1r = Zw + (long long)c * (L / 2);
  const float2* o1r = Zw + (long long)(M + c) * (L / 2);
  const float2* e2r = Zw + (long long)kb * (L / 2);
  const float2* o2r = Zw + (long long)(M + kb) * (L / 2);
  // radix-2 twiddles on O[c] and O[kb]: W_N1^c and W_N1^{-c}, or 1 and W_N1^{M/2}
  const float2 w = __ldg(a.r2w + c);
  const float2 w1 = first ? make_float2(1.f, 0.f) : w;
  const float2 w2 = first ? __ldg(a.r2w + M / 2) : conjf2(w);
  const int t = mirror_lane_butterfly<TPS>(g);
  const uint64_t pol = l2::evict_first();  // last use of the workspace
  pdl::wait_prior_grid();
  soa::C2 v[16];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = t + TPS * j;
    const float2 e1 = l2::ld_once(e1r + p, pol), e2 = l2::ld_once(e2r + p, pol);
    const float2 o1 = cmul(l2::ld_once(o1r + p, pol), w1), o2 = cmul(l2::ld_once(o2r + p, pol), w2);
    const float2 P = cadd(e1, o1), Q = csub(e1, o1), Rr = cadd(e2, o2), S = csub(e2, o2);
    // (z_a, m_a, z_b, m_b) = (V[c], V[N1-c], V[M-c], V[M+c]); first group:
    // (V[0], V[M], V[M/2], V[3M/2])
    const float2 Am = first ? Q : Rr, B = first ? Rr : S, Bm = first ? S : Q;
    split_point<MASK>(P, Am, B, Bm, first, v[j], v[15 - j]);
  }
  soa::first_stage<L, false>(v, s, t);
  __syncthreads();
  soa::stages<L, 16, false>(s, g, a.tw2x);
  pdl::launch_dependents();
  fwd_post_x2<L>(s, a, a.out + (long long)blockIdx.z * a.out_bstride, c, kb, first, g);
}

// Inverse pairing of both items into E' / O' rows: from the row IFFT u in s,
// Z(k, p) of the items' rows as in the four-step family's pairing, then
//   E'[c] = V[c] + V[M+c],      O'[c] = conj(w) (V[c] - V[M+c])
//   E'[M-c] = V[M-c] + V[N1-c], O'[M-c] = w (V[N1-c] - V[M-c])
// and for the first group E'[0], O'[0] from V[0] +- V[M], E'[M/2] = V[M/2] +
// V[3M/2], O'[M/2] = i (V[M/2] - V[3M/2]).
template <int L>
__device__ __forceinline__ void tp_inv_pair(const float4* __restrict__ s, const Dct2dArgs& a, float2* Zw, int c,
                                            int kb, bool first, int g) {
  constexpr int TPS = fft_tps(L);
  const int M = a.n1 / 2;
  float2* e1r = Zw + (long long)c * (L / 2);
  float2* o1r = Zw + (long long)(M + c) * (L / 2);
  float2* e2r = Zw + (long long)kb * (L / 2);
  float2* o2r = Zw + (long long)(M + kb) * (L / 2);
  const float2 w = __ldg(a.r2w + c);
  const uint64_t pol = l2::evict_last();  // read again by the column pass
#pragma unroll 2
  for (int r = 0; r < L / 2 / TPS; ++r) {
    const int p = g + TPS * r;
    const soa::C2 u = soa::unpack(s[soa::pidx4(p)]), wv = soa::unpack(s[soa::pidx4(L - 1 - p)]);
    const float2 zb0 = make_float2(u.re.y - wv.im.y, u.im.y + wv.re.y);  // V[kb]
    const float2 zb1 = make_float2(u.re.y + wv.im.y, wv.re.y - u.im.y);  // V[mirror of kb]
    const float2 za0 = first ? make_float2(u.re.x, wv.re.x) : make_float2(u.re.x - wv.im.x, u.im.x + wv.re.x);
    const float2 za1 = first ? make_float2(u.im.x, wv.im.x) : make_float2(u.re.x + wv.im.x, wv.re.x - u.im.x);
    const float2 x1 = first ? za1 : zb1;  // V[c + M]
    const float2 x2 = first ? zb1 : za1;  // V[kb + M]
    const float2 d1 = csub(za0, x1);
    const float2 d2 = csub(zb0, x2);
    const float2 o1 = first ? d1 : cmulc(d1, w);
    const float2 o2 = first ? make_float2(-d2.y, d2.x) : cmul(make_float2(-d2.x, -d2.y), w);
    l2::st(e1r + p, cadd(za0, x1), pol);
    l2::st(o1r + p, o1, pol);
    l2::st(e2r + p, cadd(zb0, x2), pol);
    l2::st(o2r + p, o2, pol);
  }
}

// STAGED: the group's (up to) four input rows are first copied whole into its
// shared buffer by contiguous bulk copies (one mbarrier per group, bounded
// wait as in the column pass), so the preprocess reads each value from shared
// memory instead of twice from global memory (at k2 and at N2 - k2); the
// buffer (17 L bytes) holds the 16 L bytes of the rows until the first FFT
// stage overwrites it.  Device buffers only.

template <int L, bool MAPPED, bool STAGED, bool NARROW>
__global__ void __launch_bounds__(TpRows<L, NARROW>::THREADS, TpRows<L, NARROW>::MINB) k_tp_rows_inv(Dct2dArgs a) {
  using R = TpRows<L, NARROW>;
  extern __shared__ float4 sxti[];
  const int pi = threadIdx.x / R::TPS, g = threadIdx.x % R::TPS;
  float4* s = sxti + pi * R::LP;
  const int M = a.n1 / 2;
  const int c = blockIdx.x * R::NP + pi;
  const bool first = (c == 0);
  const int kb = tp_item_b(c, M);
  const float* C = a.in + (long long)blockIdx.z * a.in_bstride;
  const InvRows A = inv_rows_of(a, C, c, L), B = inv_rows_of(a, C, kb, L);
  soa::C2 v[16];
  if constexpr (STAGED) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(sxti + R::NP * R::LP) + pi;
    int* flag = reinterpret_cast<int*>(reinterpret_cast<uint64_t*>(sxti + R::NP * R::LP) + R::NP);
    float* st = reinterpret_cast<float*>(s);
    if (threadIdx.x == 0) *flag = 1;
    if (g == 0) {
      tma::bar_init(bar, 1);
      tma::fence_barrier_init();
    }
    pdl::wait_prior_grid();
    __syncthreads();
    if (g == 0) {
      const float* src[4] = {A.ra, A.rb, B.ra, B.rb};  // rb rows are never null
      uint32_t bytes = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) bytes += src[i] ? L * (uint32_t)sizeof(float) : 0u;
      tma::bar_expect_tx(bar, bytes);
      const uint64_t pol = l2::evict_first();  // the input is streamed in
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (src[i]) tma::bulk_load(st + i * L, src[i], L * (uint32_t)sizeof(float), bar, pol);
      const uint32_t polls = a.polls ? a.polls : tma::kDefaultPolls;
      if (!tma::bar_wait_from_issue(bar, 0, polls)) {
        atomicExch(a.err, 1);
        tma::bar_wait(bar, 0, tma::kDefaultPolls);  // the copies must land before the CTA exits
        *flag = 0;
      }
    }
    __syncthreads();
    if (!*flag) return;
    tma::test_wait(bar, 0);  // completed: every thread observes the copied rows
    const InvRows As{A.ra ? st : nullptr, st + L}, Bs{B.ra ? st + 2 * L : nullptr, st + 3 * L};
    if (first)
      inv_pre_x2<L, MAPPED, true, true>(a, As, Bs, c, kb, g, v);
    else
      inv_pre_x2<L, MAPPED, false, true>(a, As, Bs, c, kb, g, v);
    __syncthreads();  // the first stage overwrites the staged rows
  } else {
    pdl::wait_prior_grid();
    if (first)
      inv_pre_x2<L, MAPPED, true>(a, A, B, c, kb, g, v);
    else
      inv_pre_x2<L, MAPPED, false>(a, A, B, c, kb, g, v);
  }
  soa::first_stage<L, true>(v, s, g);
  __syncthreads();
  soa::stages<L, 16, true>(s, g, a.tw2x);
  pdl::launch_dependents();
  tp_inv_pair<L>(s, a, a.work + (long long)blockIdx.z * a.work_bstride, c, kb, first, g);
}

}  // namespace gbdct
