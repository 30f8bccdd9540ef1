// pass2_inv_rows.cu - instances of k_inv_rows2<L> (two-sequence pass) for L = 16 .. 8192.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_PAIR_RUNNER(run_inv_rows2, k_inv_rows2)
}  // namespace gbdct
