// Packed-pair t-side sweep kernels for t-planes 32 wide, half-widths 1..6.
#include "tside.cuh"

namespace fpca_sweep {

bool tsweep_c32_a(FPCA_TSWEEP_PARAMS) { return tsweep_launch_range<32, 1, 6>(FPCA_TSWEEP_ARGS); }

}  // namespace fpca_sweep
