// Multi-problem pass kernels (see multi.h): the work list of one launch
// spans the members of slots 288, 432 and 576; each CTA takes one item and
// runs the length-specialised body of its member's extent (fast_kernels.cuh)
// with RP = BS / TPT row pairs, or CBW = BS / TPT columns, per item.
#pragma once
#include <algorithm>

#include "fast_kernels.cuh"
#include "multi.h"

namespace qpat {

// Resident CTAs per SM the kernels are compiled for: row blocks of 144
// threads four, of 288 two; column blocks of 288 two, of 576 one.
__host__ __device__ constexpr int multi_row_minb(int bs) { return bs <= 144 ? 4 : 2; }
__host__ __device__ constexpr int multi_col_minb(int bs) { return bs <= 288 ? 2 : 1; }

template <int PH, int BS>
constexpr size_t multi_row_smem() {
  constexpr size_t a = row_fast_st_smem<float, 288, PH, BS / 48>();
  constexpr size_t b = row_fast_st_smem<float, 432, PH, BS / 72>();
  constexpr size_t c = row_fast_st_smem<float, 576, PH, BS / 72>();
  constexpr size_t m = a > b ? a : b;
  return m > c ? m : c;
}
template <int PH, int BS>
constexpr size_t multi_col_smem() {
  constexpr size_t a = col_fast_smem<float, 288, PH, BS / 48>();
  constexpr size_t b = col_fast_smem<float, 432, PH, BS / 72>();
  constexpr size_t c = col_fast_smem<float, 576, PH, BS / 72>();
  constexpr size_t m = a > b ? a : b;
  return m > c ? m : c;
}

// One work item per CTA (blockIdx.x; reversed when m.reverse).  A grid-stride
// loop over the items would keep each CTA resident across items, but ptxas
// then holds the radix DFTs' packed constants across iterations and spills
// about 1.4 KB per thread at 96 registers (against 48 bytes here), so the
// launch has one CTA per item and the block scheduler keeps the SMs busy.
template <int PH, int BS>
__global__ void __launch_bounds__(BS, multi_row_minb(BS)) row_multi(const __grid_constant__ MultiArgs m) {
  static_assert(BS % 48 == 0 && BS % 72 == 0, "block size must hold whole row groups of every extent");
  const int total = m.first[kMultiSlots];
  const int item = m.reverse ? total - 1 - (int)blockIdx.x : (int)blockIdx.x;
  if (item < m.first[1]) {
    row_st_body<float, 288, PH, BS / 48>(m.a[0], item / m.per[0], item % m.per[0]);
  } else if (item < m.first[2]) {
    const int loc = item - m.first[1];
    row_st_body<float, 432, PH, BS / 72>(m.a[1], loc / m.per[1], loc % m.per[1]);
  } else {
    const int loc = item - m.first[2];
    row_st_body<float, 576, PH, BS / 72>(m.a[2], loc / m.per[2], loc % m.per[2]);
  }
}

template <int PH, int BS>
__global__ void __launch_bounds__(BS, multi_col_minb(BS)) col_multi(const __grid_constant__ MultiArgs m) {
  static_assert(BS % 48 == 0 && BS % 72 == 0, "block size must hold whole column groups of every extent");
  const int total = m.first[kMultiSlots];
  const int item = m.reverse ? total - 1 - (int)blockIdx.x : (int)blockIdx.x;
  if (item < m.first[1]) {
    col_body<float, 288, PH, BS / 48>(m.a[0], item / m.per[0], item % m.per[0], m.per[0]);
  } else if (item < m.first[2]) {
    const int loc = item - m.first[1];
    col_body<float, 432, PH, BS / 72>(m.a[1], loc / m.per[1], loc % m.per[1], m.per[1]);
  } else {
    const int loc = item - m.first[2];
    col_body<float, 576, PH, BS / 72>(m.a[2], loc / m.per[2], loc % m.per[2], m.per[2]);
  }
}

// Shared-memory attribute and launch of one (phase, block size).
template <int PH, int BS>
cudaError_t multi_row_attr() {
  static_assert(multi_row_smem<PH, BS>() <= 227 * 1024, "multi row pass above 227 KB of shared memory");
  return cudaFuncSetAttribute(row_multi<PH, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)multi_row_smem<PH, BS>());
}
template <int PH, int BS>
cudaError_t multi_col_attr() {
  static_assert(multi_col_smem<PH, BS>() <= 227 * 1024, "multi column pass above 227 KB of shared memory");
  return cudaFuncSetAttribute(col_multi<PH, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)multi_col_smem<PH, BS>());
}
template <int PH, int BS>
int multi_row_occ() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, row_multi<PH, BS>, BS, multi_row_smem<PH, BS>());
  return n;
}
template <int PH, int BS>
int multi_col_occ() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, col_multi<PH, BS>, BS, multi_col_smem<PH, BS>());
  return n;
}

// Entry points of one row block size (one translation unit each).
template <int BS>
void launch_multi_row_bs(const MultiArgs& m, int ph, int ctas, cudaStream_t s) {
  switch (ph) {
#define QPAT_MR(P) case P: row_multi<P, BS><<<ctas, BS, multi_row_smem<P, BS>(), s>>>(m); break;
    QPAT_MR(F_R1) QPAT_MR(F_R2) QPAT_MR(F_R3) QPAT_MR(F_R3L) QPAT_MR(A_R1) QPAT_MR(A_R1L) QPAT_MR(A_R3)
    QPAT_MR(A_R5)
#undef QPAT_MR
    default: break;
  }
}
template <int BS>
cudaError_t prepare_multi_row_bs(int* occ) {
  cudaError_t e = cudaSuccess;
  int o = 1 << 20;
#define QPAT_MR(P)                                         \
  if (e == cudaSuccess) e = multi_row_attr<P, BS>();       \
  if (e == cudaSuccess) o = std::min(o, multi_row_occ<P, BS>());
  QPAT_MR(F_R1) QPAT_MR(F_R2) QPAT_MR(F_R3) QPAT_MR(F_R3L) QPAT_MR(A_R1) QPAT_MR(A_R1L) QPAT_MR(A_R3)
  QPAT_MR(A_R5)
#undef QPAT_MR
  *occ = o;
  return e;
}
template <int BS>
void launch_multi_col_bs(const MultiArgs& m, int ph, int ctas, cudaStream_t s) {
  switch (ph) {
#define QPAT_MC(P) case P: col_multi<P, BS><<<ctas, BS, multi_col_smem<P, BS>(), s>>>(m); break;
    QPAT_MC(F_C1) QPAT_MC(F_C2) QPAT_MC(F_C3) QPAT_MC(A_C2) QPAT_MC(A_C4) QPAT_MC(A_C6)
#undef QPAT_MC
    default: break;
  }
}
template <int BS>
cudaError_t prepare_multi_col_bs(int* occ) {
  cudaError_t e = cudaSuccess;
  int o = 1 << 20;
#define QPAT_MC(P)                                         \
  if (e == cudaSuccess) e = multi_col_attr<P, BS>();       \
  if (e == cudaSuccess) o = std::min(o, multi_col_occ<P, BS>());
  QPAT_MC(F_C1) QPAT_MC(F_C2) QPAT_MC(F_C3) QPAT_MC(A_C2) QPAT_MC(A_C4) QPAT_MC(A_C6)
#undef QPAT_MC
  *occ = o;
  return e;
}

#define QPAT_MULTI_ROWS(BS)                                                                       \
  template void launch_multi_row_bs<BS>(const MultiArgs&, int, int, cudaStream_t);               \
  template cudaError_t prepare_multi_row_bs<BS>(int*);
#define QPAT_MULTI_COLS(BS)                                                                       \
  template void launch_multi_col_bs<BS>(const MultiArgs&, int, int, cudaStream_t);               \
  template cudaError_t prepare_multi_col_bs<BS>(int*);

}  // namespace qpat
