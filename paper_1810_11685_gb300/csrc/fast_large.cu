// Compile-time Stockham propagation passes for FFT extents 1024 and 1080 (see fast_kernels.cuh).
#include "fast_kernels.cuh"
namespace qpat {
QPAT_FAST_LENGTH(1024)
QPAT_FAST_LENGTH(1080)
}  // namespace qpat
