// Compile-time Stockham 3D propagation passes for FFT extent 288 (see fast3_kernels.cuh).
#include "fast3_kernels.cuh"
namespace qpat {
QPAT_FAST3_LENGTH(288)
}  // namespace qpat
