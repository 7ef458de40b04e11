// Compile-time Stockham propagation passes for the small FFT extents 24, 40, 48, 54, 56
// (see fast_kernels.cuh).
#include "fast_kernels.cuh"
namespace qpat {
QPAT_FAST_LENGTH(24)
QPAT_FAST_LENGTH(40)
QPAT_FAST_LENGTH(48)
QPAT_FAST_LENGTH(54)
QPAT_FAST_LENGTH(56)
}  // namespace qpat
