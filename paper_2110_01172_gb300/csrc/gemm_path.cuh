// gemm_path.cuh - the split-BF16 DFT-GEMM precision mode of a 2D plan.
//
// The separable definition X = C1 x C2^T (Eq. 2d-dct-definition; C[k, j] =
// cos(pi k (2j+1) / 2N)) and its inverse x = D1 X D2^T (D = (2/N) C^T diag(w),
// w_0 = 1/2) evaluated as dense products on the tensor cores: every operand v
// is split into bf16 parts hi = bf16(v), lo = bf16(v - hi), and each product
// A B is accumulated in FP32 as hi_A hi_B + hi_A lo_B + lo_A hi_B (the lo lo
// term, ~2^-18 relative, is dropped).  The matrices are generated in FP64 from
// integer-reduced angles and split once; x is split by a kernel per call, and
// the first product's epilogue writes the intermediate already split and
// transposed as the second product's operand.  Both products run in the
// hand-written tcgen05 kernel of tc_gemm.cuh (TMA-staged bf16 tiles, the
// three split products accumulated in one FP32 tensor-memory accumulator):
// three launches per call.  The error is that of the split (about 5e-6
// relative in L2), stated per result by the tests rather than held to the FP32
// tolerance.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbdct.h"

namespace gbdct {

struct GemmPath;

// kGemmMinSide <= n1, n2 <= kGemmMaxSide (powers of two); batch transforms
// stored back to back.  `err` is the plan's device error word (bounded waits
// that gave up set it).
constexpr int kGemmMinSide = 128;
constexpr int kGemmMaxSide = 2048;
GemmPath* gemm_create(int n1, int n2, int batch, int* err, gbdct_status* st);
// Bound (polls) of every device-side wait of the kernels; 0 restores the default.
void gemm_set_wait_polls(GemmPath* g, uint32_t polls);
gbdct_status gemm_exec(GemmPath* g, bool inverse, const float* in, float* out, cudaStream_t s);
size_t gemm_workspace_bytes(const GemmPath* g);
void gemm_destroy(GemmPath* g);

}  // namespace gbdct
