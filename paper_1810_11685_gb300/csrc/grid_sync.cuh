// Grid-wide barrier with a bounded wait, for cooperative launches.
//
// Thread 0 of each CTA arrives on a counter; the last CTA to arrive resets
// the counter and advances a generation word, which the others wait on.  A
// wait gives up after `limit_ns` nanoseconds of device time (globaltimer):
// the CTA records QPAT_ETIMEOUT (5) in *status and the barrier reports
// failure to every thread of the CTA, which must then leave the kernel.  The
// counter and generation words must be zero when the launch starts (the host
// clears them on the launch stream), and the grid must be co-resident
// (cudaLaunchCooperativeKernel checks that).
#pragma once
#include <cuda_runtime.h>

namespace qpat {

struct GridBar {
  unsigned* count;          // arrivals in the present generation
  unsigned* gen;            // generation, advanced by the last arrival
  int* status;              // 0, or 5 (QPAT_ETIMEOUT) once any wait gave up
  unsigned long long limit_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every thread of every CTA calls it; returns false (in every thread of the
// CTA) when the wait gave up or an earlier wait of the grid already had.
__device__ __forceinline__ bool grid_barrier(const GridBar& b) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
    int good = 1;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned g = ld_acquire_u32(b.gen);
    __threadfence();                                   // this CTA's writes before its arrival
    const unsigned prev = atomicAdd(b.count, 1u);
    if (prev == nblocks - 1) {
      *b.count = 0u;
      __threadfence();
      st_release_u32(b.gen, g + 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(b.gen) == g) {
        if (global_ns() - t0 > b.limit_ns || *((volatile int*)b.status) != 0) {
          good = 0;
          atomicExch(b.status, 5);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace qpat
