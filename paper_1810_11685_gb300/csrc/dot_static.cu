// qpat_dot_noalloc: the FP64 compensated inner product of qpat_dot with its
// scratch space in a fixed device array instead of context memory.
//
// Who needs it: code that must not allocate device memory at the point of
// the call -- for example an outer optimisation loop running under a memory
// pool that is frozen after set-up, a host framework that owns every device
// allocation itself, or an inner Krylov loop where a cudaMalloc would
// synchronise the device -- and that has no qpat context at hand.  The
// caller passes its inputs and an output array; this file owns the only
// scratch (the per-block partial sums).
//
// The scratch is a file-scope __device__ array of kNoAllocMaxBatch problems
// (512 KiB); every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device, with that device current, looks the address up
// with cudaGetSymbolAddress and caches it; make that first call before any
// stream capture.  All calls share the one array: calls that may overlap on
// the GPU (different streams, or different host threads) race on it and
// must be ordered by the caller.  Nothing has to start at zero: each call
// overwrites every partial it later reads.
#include <mutex>
#include <string>

#include "qpat.h"
#include "qpat_internal.h"

namespace {

constexpr int kNoAllocMaxBatch = 64;
constexpr int kMaxDevices = 64;

// [kNoAllocMaxBatch][kPartials][4] doubles
__device__ __align__(256) double g_dot_scratch[kNoAllocMaxBatch * qpat::kPartials * 4];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
thread_local std::string g_noalloc_err;

qpat_status noalloc_fail(qpat_status st, const std::string& msg) {
  g_noalloc_err = msg;
  return st;
}

}  // namespace

extern "C" const char* qpat_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" qpat_status qpat_dot_noalloc(int prec, int batch, long long len, const void* a, const void* b,
                                        double* out, void* stream) {
  if (prec != QPAT_FP32 && prec != QPAT_FP64) return noalloc_fail(QPAT_EINVAL, "unknown precision");
  if (batch < 1 || batch > kNoAllocMaxBatch)
    return noalloc_fail(QPAT_EINVAL, "qpat_dot_noalloc: batch " + std::to_string(batch) +
                                         " outside 1.." + std::to_string(kNoAllocMaxBatch));
  if (len < 0 || !a || !b || !out) return noalloc_fail(QPAT_EINVAL, "qpat_dot_noalloc: bad arguments");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(QPAT_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(QPAT_EINVAL, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_dot_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(QPAT_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == QPAT_FP32)
    e = qpat::dot_compensated<float>(batch, len, (const float*)a, (const float*)b, (double*)scratch, out, s);
  else
    e = qpat::dot_compensated<double>(batch, len, (const double*)a, (const double*)b, (double*)scratch, out, s);
  if (e != cudaSuccess) return noalloc_fail(QPAT_ECUDA, std::string("dot kernels: ") + cudaGetErrorString(e));
  return QPAT_OK;
}
