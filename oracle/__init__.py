"""FP64 CPU oracle for the binned local linear FPCA smoother (test infrastructure).

This package is test infrastructure only. It is the plain, slow, obviously
correct statement of what the CUDA path computes, written from the paper
(Chen & Jiang, "Multi-dimensional Functional Principal Component Analysis",
Sections 2-3). Only the test suite, the smoke check and the benchmark's
CPU-baseline arm may import it; the library path never does, and it shares no
code with the CUDA sources.

Modules
  smoother  binning (Section 3.2), local linear smoothers Eq. (2.3)-(2.4),
            per-point solve and status
  eigen     matrixisation and rescaling (Section 3.1, Eq. 3.1) and the random
            projection (Section 3.4)
  block     the covariance smoother at chosen output pairs (rows, tiles) from
            the data, for grids whose P x P bins are too large to hold
  grid      the covariance smoother on whole grids of up to 64 x 64 nodes
            (the moments as band-matrix products, a stacked solve)
  variance  the noise variance of Eq. (2.5)-(2.6)
  scores    PACE scores (Eq. 2.7), scores by integration, reconstruction
  cv        cross-validation of the covariance bandwidth (Section 3.3)
  mlp       the bandwidth-proposal network (forward, manual backward, AdamW)
"""
from . import smoother, eigen, cv, block, grid, variance, scores  # noqa: F401
