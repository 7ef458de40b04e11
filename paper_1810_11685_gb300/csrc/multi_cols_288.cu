// Persistent multi-problem column passes, 288-thread blocks (see multi_kernels.cuh).
#include <algorithm>

#include "multi_kernels.cuh"
namespace qpat {
QPAT_MULTI_COLS(288)
}  // namespace qpat
