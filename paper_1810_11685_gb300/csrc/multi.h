// Multi-problem propagation passes (FP32, 2D): one launch per pass kind
// serves several contexts of different FFT extents at once -- the problems of
// an inexact-Newton inner loop on grids of uneven size.
//
// A launch covers a work list of (member, problem, tile) items: for a row
// pass a tile is RP pairs of grid rows, for a column pass CBW adjacent
// half-spectrum columns.  CTA i takes item i (or total - 1 - i) and runs the
// same length-specialised body as the single-context passes, so a member's
// results are bit for bit those of its own passes.  Members sit in slots by
// extent; each slot holds the member's PropArgs (with this launch's time
// index and flags) by value in the kernel parameters.
#pragma once
#include "qpat_internal.h"

namespace qpat {

constexpr int kMultiSlots = 3;
// FFT extent of each slot (square grids: nx = ny = extent)
__host__ __device__ constexpr int multi_extent(int slot) { return slot == 0 ? 288 : slot == 1 ? 432 : 576; }
// threads per transform of each extent (the length over its smallest radix)
__host__ __device__ constexpr int multi_tpt(int slot) { return slot == 0 ? 48 : 72; }
inline int multi_slot_of(int L) {
  for (int s = 0; s < kMultiSlots; ++s)
    if (multi_extent(s) == L) return s;
  return -1;
}

// Block sizes the kernels are built for (each a multiple of 48 and 72).
constexpr int kMultiRowBlocks[2] = {144, 288};
constexpr int kMultiColBlocks[2] = {288, 576};

struct MultiArgs {
  PropArgs<float> a[kMultiSlots];   // slot s is used when first[s + 1] > first[s]
  int first[kMultiSlots + 1];       // work-item offsets; first[kMultiSlots] = total
  int per[kMultiSlots];             // items per problem
  int reverse;                      // 1: hand out items from the last (largest extent) down
};

// Tiles per problem of slot s for a block of bs threads.
inline int multi_row_tiles(int slot, int bs, int ny) {
  const int rp = bs / multi_tpt(slot);
  return (ny / 2 + rp - 1) / rp;
}
inline int multi_col_tiles(int slot, int bs, int nxh) {
  const int cbw = bs / multi_tpt(slot);
  return (nxh + cbw - 1) / cbw;
}

// Launch pass `phase` over the work list: `ctas` (= the item count) CTAs of bs threads.
void launch_multi_row(const MultiArgs& m, int phase, int bs, int ctas, cudaStream_t s);
void launch_multi_col(const MultiArgs& m, int phase, int bs, int ctas, cudaStream_t s);
// Dynamic shared-memory limits of every multi kernel (outside any capture);
// returns a cudaError_t.
int multi_prepare();
// Largest number of CTAs of the (row or column) pass kernel of block size bs
// resident on one SM at once (the minimum over the pass kinds).
int multi_resident_per_sm(bool row, int bs);

}  // namespace qpat
