// pass_inv_cols.cu - instances of k_inv_cols<L> for L = 2 .. 16384 and their launcher.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_RUNNER(run_inv_cols, k_inv_cols)
}  // namespace gbdct
