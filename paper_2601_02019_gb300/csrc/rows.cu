// FP64 squared row norms of FP32 rows in host or device memory (the scalar
// bookkeeping of the P5 and sliding-window runtimes runs on the host).
#include <vector>

#include "kernels.cuh"

namespace as {

namespace {

// ||row||^2 in FP64, one warp per row.
__global__ void row_norm2_kernel(const float* rows, long long ld, long long n, int d, double* out) {
  const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const float* r = rows + i * ld;
  double s = 0.0;
  for (int c = lane; c < d; c += 32) {
    const double v = (double)r[c];
    s += v * v;
  }
  s = warp_sum(s);
  if (lane == 0) out[i] = s;
}

bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

as_status row_norms_f64(const float* rows, long long n, long long ld, int d, cudaStream_t s, double* out) {
  if (n <= 0) return AS_OK;
  if (!on_device(rows)) {
    for (long long i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int c = 0; c < d; ++c) {
        const double v = (double)rows[i * ld + c];
        acc += v * v;
      }
      out[i] = acc;
    }
    return AS_OK;
  }
  double* dn = nullptr;
  AS_CUDA_TRY(cudaMalloc((void**)&dn, (size_t)n * sizeof(double)));
  row_norm2_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(rows, ld, n, d, dn);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dn, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dn);
  if (e != cudaSuccess) {
    as_note_cuda_error(e, __FILE__, __LINE__);
    return as_from_cuda(e);
  }
  return AS_OK;
}

}  // namespace as
