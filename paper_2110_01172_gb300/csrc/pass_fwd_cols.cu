// pass_fwd_cols.cu - instances of k_fwd_cols<L> for L = 2 .. 16384 and their launcher.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_RUNNER(run_fwd_cols, k_fwd_cols)
}  // namespace gbdct
