// Strided SIMT GEMM used by the FP32-plain form of the d-side products and by
// the FP64 G-space products:
//     Out(m, n) = alpha * sum_k A(m, k) B(k, n) + beta * Out(m, n)
// with A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn] and
// Out(m, n) = Out[m*som + n*son], so transposes are expressed by strides.
//
// FP32 operands: products are accumulated in FP32 over chunks of 64 along k
// and the chunk sums are combined in FP64 (keeps the accumulation error near
// the FP32 storage error for k up to several thousand).  FP64 operands:
// FP64 throughout.
#include "kernels.cuh"

namespace as {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, CHUNK_TILES = 4;

template <typename T>
struct Acc;
template <>
struct Acc<float> { using type = float; };
template <>
struct Acc<double> { using type = double; };

template <typename TA, typename TB, typename TO>
__global__ void __launch_bounds__(256) gemm_strided_kernel(
    int M, int N, int K, const TA* __restrict__ A, long long sam, long long sak,
    const TB* __restrict__ B, long long sbk, long long sbn, TO* __restrict__ O, long long som,
    long long son, double alpha, double beta) {
  using TC = typename std::conditional<std::is_same<TA, float>::value && std::is_same<TB, float>::value,
                                       float, double>::type;
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  double acc[4][4];
  TC part[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.0; part[a][b] = TC(0); }
  int tiles = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    // load A tile (BM x BK) and B tile (BK x BN): 1024 elements each, 4 per thread
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int idx = tid + t * 256;
      // A: choose the fast index by stride so that consecutive threads read
      // consecutive addresses when possible
      int mm, kk;
      if (sak == 1) { kk = idx % BK; mm = idx / BK; } else { mm = idx % BM; kk = idx / BM; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (TC)A[(long long)gm * sam + (long long)gk * sak] : TC(0);
      int nn, kb;
      if (sbn == 1) { nn = idx % BN; kb = idx / BN; } else { kb = idx % BK; nn = idx / BK; }
      const int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < N && gk2 < K) ? (TC)B[(long long)gk2 * sbk + (long long)gn * sbn] : TC(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TC a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][ty + 16 * t]; b[t] = Bs[kk][tx + 16 * t]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
    }
    __syncthreads();
    if (std::is_same<TC, float>::value) {
      if (++tiles == CHUNK_TILES) {
        tiles = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) { acc[i][j] += (double)part[i][j]; part[i][j] = TC(0); }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] += (double)part[i][j];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      TO* o = O + (long long)gm * som + (long long)gn * son;
      double v = alpha * acc[i][j];
      if (beta != 0.0) v += beta * (double)(*o);
      *o = (TO)v;
    }
  }
}

}  // namespace

template <typename TA, typename TB, typename TO>
as_status gemm_strided(cudaStream_t s, int M, int N, int K, const TA* A, long long sam, long long sak,
                       const TB* B, long long sbk, long long sbn, TO* O, long long som, long long son,
                       double alpha, double beta) {
  if (M <= 0 || N <= 0) return AS_OK;
  if (K <= 0) {
    // Out = beta * Out: only used with beta == 0 here
    K = 0;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  gemm_strided_kernel<TA, TB, TO><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, O, som, son,
                                                       alpha, beta); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

template as_status gemm_strided<float, float, float>(cudaStream_t, int, int, int, const float*, long long,
                                                     long long, const float*, long long, long long, float*,
                                                     long long, long long, double, double);
template as_status gemm_strided<float, float, double>(cudaStream_t, int, int, int, const float*, long long,
                                                      long long, const float*, long long, long long,
                                                      double*, long long, long long, double, double);
template as_status gemm_strided<double, double, double>(cudaStream_t, int, int, int, const double*,
                                                        long long, long long, const double*, long long,
                                                        long long, double*, long long, long long, double,
                                                        double);
template as_status gemm_strided<double, float, float>(cudaStream_t, int, int, int, const double*, long long,
                                                      long long, const float*, long long, long long, float*,
                                                      long long, long long, double, double);
template as_status gemm_strided<float, double, float>(cudaStream_t, int, int, int, const float*, long long,
                                                      long long, const double*, long long, long long, float*,
                                                      long long, long long, double, double);
template as_status gemm_strided<float, double, double>(cudaStream_t, int, int, int, const float*, long long,
                                                       long long, const double*, long long, long long,
                                                       double*, long long, long long, double, double);
template as_status gemm_strided<double, float, double>(cudaStream_t, int, int, int, const double*,
                                                       long long, long long, const float*, long long,
                                                       long long, double*, long long, long long, double,
                                                       double);

}  // namespace as
