// Dispatch of the persistent multi-problem passes over their block sizes.
#include <mutex>

#include "multi.h"

namespace qpat {

template <int BS>
void launch_multi_row_bs(const MultiArgs& m, int ph, int ctas, cudaStream_t s);
template <int BS>
void launch_multi_col_bs(const MultiArgs& m, int ph, int ctas, cudaStream_t s);
template <int BS>
cudaError_t prepare_multi_row_bs(int* occ);
template <int BS>
cudaError_t prepare_multi_col_bs(int* occ);

namespace {
std::mutex g_mu;
bool g_ready = false;
cudaError_t g_err = cudaSuccess;
int g_occ_row[2] = {0, 0}, g_occ_col[2] = {0, 0};
}  // namespace

void launch_multi_row(const MultiArgs& m, int phase, int bs, int ctas, cudaStream_t s) {
  if (bs == 144) launch_multi_row_bs<144>(m, phase, ctas, s);
  else if (bs == 288) launch_multi_row_bs<288>(m, phase, ctas, s);
}

void launch_multi_col(const MultiArgs& m, int phase, int bs, int ctas, cudaStream_t s) {
  if (bs == 288) launch_multi_col_bs<288>(m, phase, ctas, s);
  else if (bs == 576) launch_multi_col_bs<576>(m, phase, ctas, s);
}

int multi_prepare() {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ready) return (int)g_err;
  cudaError_t e = prepare_multi_row_bs<144>(&g_occ_row[0]);
  if (e == cudaSuccess) e = prepare_multi_row_bs<288>(&g_occ_row[1]);
  if (e == cudaSuccess) e = prepare_multi_col_bs<288>(&g_occ_col[0]);
  if (e == cudaSuccess) e = prepare_multi_col_bs<576>(&g_occ_col[1]);
  g_err = e;
  g_ready = true;
  return (int)e;
}

int multi_resident_per_sm(bool row, int bs) {
  if (row) return bs == 144 ? g_occ_row[0] : bs == 288 ? g_occ_row[1] : 0;
  return bs == 288 ? g_occ_col[0] : bs == 576 ? g_occ_col[1] : 0;
}

}  // namespace qpat
