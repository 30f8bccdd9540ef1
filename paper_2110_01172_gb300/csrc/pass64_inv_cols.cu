// pass64_inv_cols.cu - instances of k_inv_cols_r64<L> (radix-64 pass) for L = 4096, 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_R64_RUNNER(run_inv_cols_r64, k_inv_cols_r64)
}  // namespace gbdct
