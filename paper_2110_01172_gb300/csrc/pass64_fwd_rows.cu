// pass64_fwd_rows.cu - instances of k_fwd_rows_r64<L> (radix-64 pass) for L = 4096, 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_R64_RUNNER(run_fwd_rows_r64, k_fwd_rows_r64)
}  // namespace gbdct
