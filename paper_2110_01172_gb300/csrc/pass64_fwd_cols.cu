// pass64_fwd_cols.cu - instances of k_fwd_cols_r64<L> (radix-64 pass) for L = 4096, 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_R64_RUNNER(run_fwd_cols_r64, k_fwd_cols_r64)
}  // namespace gbdct
