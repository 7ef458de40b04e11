// Compile-time Stockham propagation passes for FFT extent 432 (see fast_kernels.cuh).
#include "fast_kernels.cuh"
namespace qpat {
QPAT_FAST_LENGTH(432)
}  // namespace qpat
