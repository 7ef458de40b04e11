// Persistent multi-problem column passes, 576-thread blocks (see multi_kernels.cuh).
#include <algorithm>

#include "multi_kernels.cuh"
namespace qpat {
QPAT_MULTI_COLS(576)
}  // namespace qpat
