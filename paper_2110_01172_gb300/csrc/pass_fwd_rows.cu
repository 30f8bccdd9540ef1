// pass_fwd_rows.cu - instances of k_fwd_rows<L> for L = 2 .. 16384 and their launcher.
#include "dct2d_launch.cuh"

namespace gbdct {
GBDCT_DEFINE_RUNNER(run_fwd_rows, k_fwd_rows)
}  // namespace gbdct
