// Compile-time Stockham propagation passes for FFT extent 288 (see fast_kernels.cuh).
#include "fast_kernels.cuh"
namespace qpat {
QPAT_FAST_LENGTH(288)
}  // namespace qpat
