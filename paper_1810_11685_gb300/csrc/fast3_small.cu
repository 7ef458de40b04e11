// Compile-time Stockham 3D propagation passes for the small FFT extents 24 and 48
// (see fast3_kernels.cuh).
#include "fast3_kernels.cuh"
namespace qpat {
QPAT_FAST3_LENGTH(24)
QPAT_FAST3_LENGTH(48)
}  // namespace qpat
