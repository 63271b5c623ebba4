// Self-test of the bounded device waits.  Each kernel runs one of the waits
// the library's kernels use (a release flag, a grid barrier, an mbarrier
// phase) on something that nothing completes, with a short limit: the wait
// must give up, record AS_ETIMEOUT in the status word and return, leaving the
// context usable.  No wait in this file can outlive its limit.
#include "grid.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace as {
namespace {

__global__ void flag_wait_selftest(const unsigned* flag, int* status, unsigned long long limit_ns) {
  if (threadIdx.x == 0) wait_flag_ge(flag, 1u, status, limit_ns);   // nothing ever sets the flag
}

__global__ void grid_barrier_selftest(unsigned* cnt, int* status, unsigned long long limit_ns) {
  grid_barrier(cnt, gridDim.x + 1u, status, limit_ns);   // one arrival short of the target
}

__global__ void mbar_selftest(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);   // one expected arrival, which never comes
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) set_status(status, AS_ETIMEOUT);
}

}  // namespace
}  // namespace as

extern "C" as_status as_wait_selftest(int32_t kind, int32_t limit_ms, void* cuda_stream) {
  if (kind < 0 || kind > 2 || limit_ms < 1 || limit_ms > 2000) return AS_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* buf = nullptr;   // [0] flag or counter, [1] status word
  AS_CUDA_TRY(cudaMalloc((void**)&buf, 2 * sizeof(unsigned)));
  as_status st = AS_OK;
  int ds = 0;
  const unsigned long long limit = (unsigned long long)limit_ms * 1000000ull;
  int* status = reinterpret_cast<int*>(buf + 1);
  cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    if (kind == 0) as::flag_wait_selftest<<<1, 32, 0, s>>>(buf, status, limit);
    else if (kind == 1) as::grid_barrier_selftest<<<1, 32, 0, s>>>(buf, status, limit);
    else as::mbar_selftest<<<1, 32, 0, s>>>(status, limit);
    as::count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ds, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    as_note_cuda_error(e, __FILE__, __LINE__);
    st = as_from_cuda(e);
  }
  cudaFree(buf);
  return st != AS_OK ? st : (as_status)ds;
}
