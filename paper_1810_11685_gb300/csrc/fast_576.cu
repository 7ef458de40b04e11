// Compile-time Stockham propagation passes for FFT extent 576 (see fast_kernels.cuh).
#include "fast_kernels.cuh"
namespace qpat {
QPAT_FAST_LENGTH(576)
}  // namespace qpat
