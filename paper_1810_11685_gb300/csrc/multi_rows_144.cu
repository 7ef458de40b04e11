// Persistent multi-problem row passes, 144-thread blocks (see multi_kernels.cuh).
#include <algorithm>

#include "multi_kernels.cuh"
namespace qpat {
QPAT_MULTI_ROWS(144)
}  // namespace qpat
