// qpat_barrier_check: exercises the bounded grid barrier of grid_sync.cuh
// (the one the cooperative M_gamma solve uses) on its own, so that a test can
// make a wait run out without touching a solver: `absent` CTAs of the grid
// return before the first barrier, the others wait, give up after the limit
// and leave QPAT_ETIMEOUT in the status word, and the kernel ends.
#include <string>

#include "grid_sync.cuh"
#include "qpat.h"

namespace {

constexpr int kCheckThreads = 64;

// `rounds` rounds of two barriers; CTAs with index below `absent` never
// arrive.  In round r every arriving CTA adds 1 to counter[r % 2] between the
// barriers and, after the second, checks that it holds the number of arriving
// CTAs (a barrier that let a CTA through early shows as a short count).  The
// first arriving CTA clears the slot of round r - 1 for round r + 1 (every
// check of round r - 1 precedes the first barrier of round r).
__global__ void __launch_bounds__(kCheckThreads) barrier_check_kernel(qpat::GridBar gb, int rounds, int absent,
                                                                      unsigned* counter, int* mismatch) {
  if ((int)blockIdx.x < absent) return;
  const unsigned arriving = gridDim.x - (unsigned)absent;
  for (int r = 0; r < rounds; ++r) {
    if (!qpat::grid_barrier(gb)) return;
    if (threadIdx.x == 0) {
      if (r > 0 && (int)blockIdx.x == absent) counter[(r - 1) & 1] = 0u;
      atomicAdd(&counter[r & 1], 1u);
    }
    if (!qpat::grid_barrier(gb)) return;
    if (threadIdx.x == 0 && atomicAdd(&counter[r & 1], 0u) != arriving) atomicExch(mismatch, 1);
  }
}

}  // namespace

extern "C" qpat_status qpat_barrier_check(int blocks, int rounds, int absent, double limit_s, void* stream,
                                          int* status) {
  if (!status) return QPAT_EINVAL;
  *status = -1;
  if (blocks < 1 || rounds < 1 || absent < 0 || absent >= blocks || !(limit_s > 0.0) || limit_s > 10.0)
    return QPAT_EINVAL;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QPAT_ECUDA;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return QPAT_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QPAT_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_check_kernel, kCheckThreads, 0) != cudaSuccess)
    return QPAT_ECUDA;
  if ((long long)blocks > (long long)sms * per_sm) return QPAT_EINVAL;   // must be co-resident
  cudaStream_t s = (cudaStream_t)stream;
  // [0] arrivals [1] generation [2] status [3] mismatch [4..5] counters
  int* buf = nullptr;
  if (cudaMalloc(&buf, 8 * sizeof(int)) != cudaSuccess) return QPAT_ENOMEM;
  qpat_status st = QPAT_OK;
  int host[8] = {};
  qpat::GridBar gb{reinterpret_cast<unsigned*>(buf), reinterpret_cast<unsigned*>(buf + 1), buf + 2,
                   (unsigned long long)(limit_s * 1e9)};
  unsigned* counter = reinterpret_cast<unsigned*>(buf + 4);
  int* mismatch = buf + 3;
  void* args[] = {&gb, &rounds, &absent, &counter, &mismatch};
  if (cudaMemsetAsync(buf, 0, 8 * sizeof(int), s) != cudaSuccess ||
      cudaLaunchCooperativeKernel((const void*)barrier_check_kernel, dim3(blocks), dim3(kCheckThreads), args, 0, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(host, buf, 8 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    st = QPAT_ECUDA;
  } else if (host[2] != 0) {
    st = QPAT_ETIMEOUT;
  } else if (host[3] != 0) {
    st = QPAT_ECUDA;                                       // a barrier let a CTA through early
  }
  cudaFree(buf);
  *status = (int)st;
  return st;
}
