// pass_inv_rows.cu - instances of k_inv_rows<L> for L = 2 .. 16384 and their launcher.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_RUNNER(run_inv_rows, k_inv_rows)
}  // namespace gbdct
