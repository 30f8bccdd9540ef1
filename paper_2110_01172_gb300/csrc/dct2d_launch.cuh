// dct2d_launch.cuh - host-side launchers of the 2D passes (one per pass kind).
//
// Each pass is compiled once per power-of-two FFT length L = 2 .. 16384 in its
// own translation unit; these launchers map the runtime log2(L) to the
// template instance.  `prepare` only raises the kernel's dynamic shared-memory
// limit (done once at plan creation), otherwise the kernel is launched.
#pragma once

#include <cuda_runtime.h>

#include "dct2d_kernels.cuh"

namespace gbdct {

constexpr int kMinLog2 = 1;
constexpr int kMaxLog2 = 14;

inline int seq_threads(int L, int seq_per_cta) { return seq_per_cta * fft_tps(L); }
inline size_t seq_smem_bytes(int L, int seq_per_cta) {
  return (size_t)seq_per_cta * (size_t)pad_len(L) * sizeof(float2);
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
