// Persistent multi-problem row passes, 288-thread blocks (see multi_kernels.cuh).
#include <algorithm>

#include "multi_kernels.cuh"
namespace qpat {
QPAT_MULTI_ROWS(288)
}  // namespace qpat
