// dct2d_launch.cuh - host-side launchers of the 2D passes (one per pass kind).
//
// Each pass is compiled once per power-of-two FFT length L = 2 .. 16384 in its
// own translation unit; these launchers map the runtime log2(L) to the
// template instance.  `prepare` only raises the kernel's dynamic shared-memory
// limit (done once at plan creation), otherwise the kernel is launched.
#pragma once

#include <cuda_runtime.h>

#include "dct2d_kernels.cuh"
#include "dct2d_pair_kernels.cuh"
#include "dct2d_fs2_kernels.cuh"

namespace gbdct {

constexpr int kMinLog2 = 1;
constexpr int kMaxLog2 = 14;

inline int seq_threads(int L, int seq_per_cta) { return seq_per_cta * fft_tps(L); }
inline size_t seq_smem_bytes(int L, int seq_per_cta) {
  return (size_t)seq_per_cta * (size_t)pad_len<float2>(L) * sizeof(float2);
}

// Sequences per CTA: enough to give the CTA ~512 threads (1024 at L = 16384,
// where one sequence already needs 1024 threads), capped by what exists.
inline int choose_seq_per_cta(int L, int nseq) {
  const int target = (L >= 16384) ? 1024 : 512;
  int b = target / fft_tps(L);
  if (b < 1) b = 1;
  if (b > nseq) b = nseq;
  return b;
}

cudaError_t run_fwd_cols(int log2L, const Dct2dArgs& a, dim3 grid, cudaStream_t s, bool prepare);
cudaError_t run_fwd_rows(int log2L, const Dct2dArgs& a, dim3 grid, cudaStream_t s, bool prepare);
cudaError_t run_inv_rows(int log2L, const Dct2dArgs& a, dim3 grid, cudaStream_t s, bool prepare);
cudaError_t run_inv_cols(int log2L, const Dct2dArgs& a, dim3 grid, cudaStream_t s, bool prepare);

// Two-sequence (float4) passes for 16 <= L <= 8192: `npairs` sequence pairs
// per transform, `batch` transforms (grid.y).
cudaError_t run_fwd_cols2(int log2L, const Dct2dArgs& a, int npairs, int batch, cudaStream_t s, bool prepare);
cudaError_t run_fwd_rows2(int log2L, const Dct2dArgs& a, int npairs, int batch, cudaStream_t s, bool prepare);
cudaError_t run_inv_rows2(int log2L, const Dct2dArgs& a, int npairs, int batch, cudaStream_t s, bool prepare);
cudaError_t run_inv_cols2(int log2L, const Dct2dArgs& a, int npairs, int batch, cudaStream_t s, bool prepare);
// Four-step family: N1 in {256, ..., 8192}, N2 in {256, ..., 16384}.  One call
// launches the whole forward (C1, C2, row pass) or inverse (row pass, C2', C1').
cudaError_t run_fs2(int log2N1, int log2N2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s,
                    bool prepare);
cudaError_t run_fs2_col(int lg1, int kind, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare);
constexpr int kFs2MinLog2N1 = 8, kFs2MaxLog2N1 = 13, kFs2MinLog2N2 = 8, kFs2MaxLog2N2 = 14;
// Default four-step split N1 = A * B (the autotuner may choose another one,
// gbdct_plan_create_tuned); A = 16 at N1 = 2048 measured faster than 32 or 64.
inline void fs2_split(int log2N1, int* A, int* B) {
  const int n1 = 1 << log2N1;
  *A = (n1 == 2048) ? 16 : (n1 >= 4096) ? 64 : (n1 >= 512 ? 32 : 16);
  *B = n1 / *A;
}

// Two-pass family: N1 in {128, ..., 8192}, N2 in {128, ..., 8192}.  One call
// launches the whole forward (column pass, row pass) or inverse (row pass,
// column pass).
cudaError_t run_tp(int log2N1, int log2N2, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s,
                   bool prepare);
cudaError_t run_tp_cols(int lg1, bool inverse, const Dct2dArgs& a, int batch, cudaStream_t s, bool prepare);
constexpr int kTpMinLog2N1 = 7, kTpMaxLog2N1 = 13, kTpMinLog2N2 = 7, kTpMaxLog2N2 = 13;
// Strip widths NP (column pairs per CTA) the two-pass column pass is built
// for at half-length M: 64 to 512 threads (M/16 per pair), the strip's
// padded shared memory within 227 KB, and N2/4 float4 columns a multiple of NP.
inline bool tp_strip_ok(int M, int n2, int np) {
  const int threads = np * (M / 16);
  const size_t smem = (size_t)np * (M + M / 16) * 16;
  return np >= 1 && threads >= 64 && threads <= 512 && smem <= 227 * 1024 - 256 && (n2 / 4) % np == 0;
}

constexpr int kPairMinLog2 = 4;
constexpr int kPairMaxLog2 = 13;

template <int L>
cudaError_t launch_pair(void (*kern)(Dct2dArgs), const Dct2dArgs& a, int npairs, int batch, cudaStream_t s,
                        bool prepare) {
  using G = PairGeom<L>;
  if (prepare) {
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(kern),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  }
  const dim3 grid((npairs + G::PB - 1) / G::PB, batch);
  kern<<<grid, G::THREADS, G::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_pass(void (*kern)(Dct2dArgs), const Dct2dArgs& a, dim3 grid, cudaStream_t s,
                        bool prepare) {
  const size_t smem = seq_smem_bytes(L, a.seq_per_cta);
  if (prepare) {
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(kern),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  kern<<<grid, seq_threads(L, a.seq_per_cta), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gbdct

// Defines run_<NAME>(log2L, ...) dispatching to kernel template KERN<L>.
#define GBDCT_DEFINE_RUNNER(NAME, KERN)                                                   \
  cudaError_t NAME(int log2L, const Dct2dArgs& a, dim3 grid, cudaStream_t s, bool prep) { \
    switch (log2L) {                                                                      \
      case 1: return launch_pass<2>(KERN<2>, a, grid, s, prep);                           \
      case 2: return launch_pass<4>(KERN<4>, a, grid, s, prep);                           \
      case 3: return launch_pass<8>(KERN<8>, a, grid, s, prep);                           \
      case 4: return launch_pass<16>(KERN<16>, a, grid, s, prep);                         \
      case 5: return launch_pass<32>(KERN<32>, a, grid, s, prep);                         \
      case 6: return launch_pass<64>(KERN<64>, a, grid, s, prep);                         \
      case 7: return launch_pass<128>(KERN<128>, a, grid, s, prep);                       \
      case 8: return launch_pass<256>(KERN<256>, a, grid, s, prep);                       \
      case 9: return launch_pass<512>(KERN<512>, a, grid, s, prep);                       \
      case 10: return launch_pass<1024>(KERN<1024>, a, grid, s, prep);                    \
      case 11: return launch_pass<2048>(KERN<2048>, a, grid, s, prep);                    \
      case 12: return launch_pass<4096>(KERN<4096>, a, grid, s, prep);                    \
      case 13: return launch_pass<8192>(KERN<8192>, a, grid, s, prep);                    \
      case 14: return launch_pass<16384>(KERN<16384>, a, grid, s, prep);                  \
      default: return cudaErrorInvalidValue;                                              \
    }                                                                                     \
  }

// Defines run_<NAME>(log2L, ...) for the two-sequence kernels, L = 16 .. 8192.
#define GBDCT_DEFINE_PAIR_RUNNER(NAME, KERN)                                                        \
  cudaError_t NAME(int log2L, const Dct2dArgs& a, int np, int nb, cudaStream_t s, bool prep) {      \
    switch (log2L) {                                                                                \
      case 4: return launch_pair<16>(KERN<16>, a, np, nb, s, prep);                                 \
      case 5: return launch_pair<32>(KERN<32>, a, np, nb, s, prep);                                 \
      case 6: return launch_pair<64>(KERN<64>, a, np, nb, s, prep);                                 \
      case 7: return launch_pair<128>(KERN<128>, a, np, nb, s, prep);                               \
      case 8: return launch_pair<256>(KERN<256>, a, np, nb, s, prep);                               \
      case 9: return launch_pair<512>(KERN<512>, a, np, nb, s, prep);                               \
      case 10: return launch_pair<1024>(KERN<1024>, a, np, nb, s, prep);                            \
      case 11: return launch_pair<2048>(KERN<2048>, a, np, nb, s, prep);                            \
      case 12: return launch_pair<4096>(KERN<4096>, a, np, nb, s, prep);                            \
      case 13: return launch_pair<8192>(KERN<8192>, a, np, nb, s, prep);                            \
      default: return cudaErrorInvalidValue;                                                        \
    }                                                                                               \
  }
