// Packed-pair t-side sweep kernels for t-planes 64 wide, half-widths 1..6.
#include "tside.cuh"

namespace fpca_sweep {

bool tsweep_c64_a(FPCA_TSWEEP_PARAMS) { return tsweep_launch_range<64, 1, 6>(FPCA_TSWEEP_ARGS); }

}  // namespace fpca_sweep
