// pass2_inv_cols.cu - instances of k_inv_cols2<L> (two-sequence pass) for L = 16 .. 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_PAIR_RUNNER(run_inv_cols2, k_inv_cols2)
}  // namespace gbdct
