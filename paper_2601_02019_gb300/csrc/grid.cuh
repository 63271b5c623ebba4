// Grid-wide barrier for cooperative (co-resident) launches, with a bounded
// wait.  Arrivals are counted on a zeroed counter that only grows: the n-th
// barrier of a launch completes when the counter reaches n * gridDim.x.
#pragma once

#include "common.cuh"

namespace as {


__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread waits (bounded) until *flag >= target; false on a timeout
// (status set to AS_ETIMEOUT) or when the sticky status is already set.
__device__ __forceinline__ bool wait_flag_ge(const unsigned* flag, unsigned target, int* status,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  const unsigned long long t0 = global_ns();
  long long n = 0;
  // the sticky status and the clock are checked every 8th poll, so a poll is
  // one L2 round trip
  while (ld_acquire_u32(flag) < target) {
    if ((++n & 7) == 0) {
      if (*(volatile int*)status != 0) return false;
      if (n > kWaitMaxIters || global_ns() - t0 > limit_ns) { set_status(status, AS_ETIMEOUT); return false; }
    }
    __nanosleep(20);
  }
  return true;
}

// Returns false when this CTA gave up waiting (status set to AS_ETIMEOUT) or
// found the sticky status already set; the caller then returns, and every
// other CTA gives up at its next barrier.
__device__ __forceinline__ bool grid_barrier(unsigned* cnt, unsigned target, int* status,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ int s_ok;
  __syncwarp();   // a block barrier needs converged warps (thread 0 ran alone)
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: this CTA's writes (ordered before by __syncthreads) become
    // visible with the arrival; acquire on the loads that observe the target
    red_release_add_u32(cnt, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    long long n = 0;
    while (ld_acquire_u32(cnt) < target) {
      if ((++n & 7) == 0) {
        if (*(volatile int*)status != 0) { ok = 0; break; }
        if (n > kWaitMaxIters || global_ns() - t0 > limit_ns) { set_status(status, AS_ETIMEOUT); ok = 0; break; }
      }
      __nanosleep(20);
    }
    s_ok = ok;
  }
  __syncwarp();   // a block barrier needs converged warps (thread 0 ran alone)
  __syncthreads();
  return s_ok != 0;
}

// The arrival and bounded wait of a grid barrier, by one thread: adds one
// arrival (release) and waits until the counter reaches `target` (acquire).
// Returns false on a timeout (status set to AS_ETIMEOUT) or when the sticky
// status is already set.  The caller orders the CTA's writes before it (a
// block or warp barrier) and releases the other threads afterwards.
__device__ __forceinline__ bool grid_arrive_wait(unsigned* cnt, unsigned target, int* status,
                                                 unsigned long long limit_ns = kWaitLimitNs) {
  red_release_add_u32(cnt, 1u);
  const unsigned long long t0 = global_ns();
  long long n = 0;
  while (ld_acquire_u32(cnt) < target) {
    if ((++n & 7) == 0) {
      if (*(volatile int*)status != 0) return false;
      if (n > kWaitMaxIters || global_ns() - t0 > limit_ns) { set_status(status, AS_ETIMEOUT); return false; }
    }
    __nanosleep(20);
  }
  return true;
}

// grid_barrier with `before_arrive` run by thread 0 after the CTA barrier and
// before its arrival (e.g. publishing a per-CTA partial that the block's
// shared memory holds); the arrival releases what it wrote.
template <typename F>
__device__ __forceinline__ bool grid_barrier_then(unsigned* cnt, unsigned target, int* status, F&& before_arrive,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ int s_ok2;
  __syncwarp();   // a block barrier needs converged warps (thread 0 ran alone)
  __syncthreads();
  if (threadIdx.x == 0) {
    before_arrive();
    red_release_add_u32(cnt, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    long long n = 0;
    while (ld_acquire_u32(cnt) < target) {
      if ((++n & 7) == 0) {
        if (*(volatile int*)status != 0) { ok = 0; break; }
        if (n > kWaitMaxIters || global_ns() - t0 > limit_ns) { set_status(status, AS_ETIMEOUT); ok = 0; break; }
      }
      __nanosleep(20);
    }
    s_ok2 = ok;
  }
  __syncwarp();   // a block barrier needs converged warps (thread 0 ran alone)
  __syncthreads();
  return s_ok2 != 0;
}

}  // namespace as
