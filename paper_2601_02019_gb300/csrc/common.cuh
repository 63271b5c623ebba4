// Device-side helpers shared by the AeroSketch kernels: status codes, error
// plumbing, block reductions and the Philox4x64-10 generator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aerosketch.h"

// Records a failed CUDA call (error name, file, line) for as_last_error().
void as_note_cuda_error(cudaError_t e, const char* file, int line);
// Raise a kernel's dynamic shared memory limit on the current device to at
// least `bytes`; it is never lowered, so a launch on another host thread that
// needs less still fits (setting the attribute per launch would race).
cudaError_t as_raise_smem_limit(const void* fn, size_t bytes);

// On failure the error is recorded and the thread's last-error state is
// cleared (cudaGetLastError), so that a later launch check does not report it
// again.
#define AS_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) {                                \
      as_note_cuda_error(_e, __FILE__, __LINE__);           \
      (void)cudaGetLastError();                             \
      return as_from_cuda(_e);                              \
    }                                                       \
  } while (0)

static inline as_status as_from_cuda(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? AS_ENOMEM : AS_EDEVICE;
}

namespace as {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): a 4-word counter and a
// 2-word key, ten rounds of 64x64->128-bit multiplies with key bumps by the
// Weyl constants between rounds.  The method's random draws use
//   counter = (purpose, timestamp i, sub-index j, element >> 2),
//   key     = (seed, stream_id),
// element e of a row-major matrix taking lane e & 3 of its counter block.
// ---------------------------------------------------------------------------
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

constexpr int kPurposePiStart = 3;  // Algorithm 1, x^(0)
constexpr int kPurposeSiTest = 4;   // Algorithm 2, Pi (sub-index = doubling step j)

struct Key { uint64_t k0, k1; };

__device__ __forceinline__ void philox4x64_10(const uint64_t c[4], Key key, uint64_t out[4]) {
  uint64_t x0 = c[0], x1 = c[1], x2 = c[2], x3 = c[3];
  uint64_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint64_t hi0 = __umul64hi(kPhiloxM0, x0), lo0 = kPhiloxM0 * x0;
    const uint64_t hi1 = __umul64hi(kPhiloxM1, x2), lo1 = kPhiloxM1 * x2;
    const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// ((w >> 12) + 1/2) * 2^-52: exactly representable, strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

// The four standard normals of counter block `blk` (Box-Muller on lanes (0,1) and (2,3)).
__device__ __forceinline__ void gauss4(Key key, uint64_t purpose, uint64_t i, uint64_t j,
                                       uint64_t blk, double z[4]) {
  const uint64_t c[4] = {purpose, i, j, blk};
  uint64_t w[4];
  philox4x64_10(c, key, w);
  const double u0 = uniform52(w[0]), u1 = uniform52(w[1]);
  const double u2 = uniform52(w[2]), u3 = uniform52(w[3]);
  const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s3, &c3);
  z[0] = r01 * c1; z[1] = r01 * s1; z[2] = r23 * c3; z[3] = r23 * s3;
}

// ---------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------
// BF16 levels of a G entry for the tensor-core products: x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1), formed from x rounded to FP32.
// Each difference is exact in FP32 (a level is its operand rounded to 8 bits,
// within a factor of two of it), so no FP64 instruction is needed beyond the
// one conversion; the levels carry about 24 bits of x, as many as the FP32
// rounding keeps.
__device__ __forceinline__ void g_levels(double x, __nv_bfloat16& l0, __nv_bfloat16& l1, __nv_bfloat16& l2) {
  const float xf = __double2float_rn(x);
  l0 = __float2bfloat16_rn(xf);
  const float r1 = xf - __bfloat162float(l0);
  l1 = __float2bfloat16_rn(r1);
  l2 = __float2bfloat16_rn(r1 - __bfloat162float(l1));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the whole block; every thread gets the result.  `red` must hold
// 32 values and is reused, so calls are separated by the trailing barrier.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : red[0];
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// Kernel launches issued by this library (all sketches); defined in engine.cu.
void count_launches(int64_t n);
int64_t launches_total();

// Sticky device status: the first non-OK code wins.
__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Device waits (grid barriers, release flags, mbarriers) give up after this
// much wall time, or after an iteration count should the timer not advance,
// set AS_ETIMEOUT and return, so that a stuck wait cannot hold the GPU.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
constexpr long long kWaitMaxIters = 1LL << 26;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace as
