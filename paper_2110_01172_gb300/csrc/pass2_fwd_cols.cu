// pass2_fwd_cols.cu - instances of k_fwd_cols2<L> (two-sequence pass) for L = 16 .. 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_PAIR_RUNNER(run_fwd_cols2, k_fwd_cols2)
}  // namespace gbdct
