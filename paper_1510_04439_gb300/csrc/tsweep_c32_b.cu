// Packed-pair t-side sweep kernels for t-planes 32 wide, half-widths 7..12.
#include "tside.cuh"

namespace fpca_sweep {

bool tsweep_c32_b(FPCA_TSWEEP_PARAMS) { return tsweep_launch_range<32, 7, 12>(FPCA_TSWEEP_ARGS); }

}  // namespace fpca_sweep
