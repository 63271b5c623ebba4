// Split-K SIMT GEMM for tall-skinny products, FP32.
//
//   P[s](m, n) = sum_{k in split s} A[m*lda + k] * X[n*ldx + k]
//
// A is row-major (m x K), X holds its n-th column contiguously (K values at
// X + n*ldx), and the S partial planes are written column-major:
// P[s*plane + n*ldp + m].  Consumers sum the S planes in a fixed order, so
// results are bitwise reproducible.  The G-space products Y = G X of the
// batched iterations (G: 2l x 2l, X: 2l x N with N <= 192) and the Gram rows
// C A_blk^T of a block use it: with one 64 x 64 tile per block, splitting K
// is what gives the grid enough blocks to fill 152 SMs.
#include "kernels.cuh"

namespace as {

namespace {

constexpr int SBM = 64, SBN = 64, SBK = 32;

__global__ void __launch_bounds__(256) skinny_partial_kernel(int M, int N, int K, int klen,
                                                             const float* __restrict__ A, long long lda,
                                                             const float* __restrict__ X, long long ldx,
                                                             float* __restrict__ P, long long ldp,
                                                             long long plane) {
  __shared__ float As[SBK][SBM + 4];
  __shared__ float Xs[SBK][SBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // tx -> rows, ty -> columns
  const int m0 = blockIdx.x * SBM, n0 = blockIdx.y * SBN;
  const int s = blockIdx.z;
  const int kb = s * klen, ke = min(K, kb + klen);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += SBK) {
#pragma unroll
    for (int t = 0; t < (SBM * SBK) / 256; ++t) {
      const int idx = tid + t * 256;
      const int rr = idx / SBK, kk = idx - rr * SBK;
      const int gm = m0 + rr, gk = k0 + kk;
      As[kk][rr] = (gm < M && gk < ke) ? A[(long long)gm * lda + gk] : 0.f;
      const int gn = n0 + rr;
      Xs[kk][rr] = (gn < N && gk < ke) ? X[(long long)gn * ldx + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < SBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][tx + 16 * t]; b[t] = Xs[kk][ty + 16 * t]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int gn = n0 + ty + 16 * j;
    if (gn >= N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + tx + 16 * i;
      if (gm < M) P[(long long)s * plane + (long long)gn * ldp + gm] = acc[i][j];
    }
  }
}

// G[p][r+t] = sum_s P[s](p, t) (FP64), mirrored to G[r+t][p] for p < r.
__global__ void gram_reduce_kernel(const float* __restrict__ P, long long ldp, long long plane, int S, int mrows,
                                   int r, int b, double* G, int n2) {
  const int t = blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < mrows; p += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += (double)P[(long long)s * plane + (long long)t * ldp + p];
    G[(long long)p * n2 + r + t] = v;
    if (p < r) G[(long long)(r + t) * n2 + p] = v;
  }
}

// out[r*ldo + c] = sum_s P[s*plane + r*ldp + c] (FP64 sum, FP32 result).
__global__ void plane_sum_kernel(const float* __restrict__ P, int S, long long plane, int rows, int cols, long long ldp,
                                 float* __restrict__ out, long long ldo) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += (double)P[(long long)s * plane + (long long)r * ldp + c];
    out[(long long)r * ldo + c] = (float)v;
  }
}

}  // namespace

as_status launch_plane_sum(cudaStream_t s, const float* P, int S, long long plane, int rows, int cols, long long ldp,
                           float* out, long long ldo) {
  if (rows <= 0 || cols <= 0) return AS_OK;
  const long long tot = (long long)rows * cols;
  const int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
  plane_sum_kernel<<<blocks, 256, 0, s>>>(P, S, plane, rows, cols, ldp, out, ldo); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

int skinny_splits(int M, int N, int K) {
  const int tiles = ((M + SBM - 1) / SBM) * ((N + SBN - 1) / SBN);
  int S = (2 * 152 + tiles - 1) / tiles;
  const int kmax = std::max(1, K / 128);  // at least 128 values of K per split
  S = std::max(1, std::min(S, kmax));
  return std::min(S, 64);
}

as_status launch_skinny_partial(cudaStream_t s, int M, int N, int K, int* S, const float* A, long long lda,
                                const float* X, long long ldx, float* P, long long ldp, long long plane) {
  if (M <= 0 || N <= 0) return AS_OK;
  int klen = (K + *S - 1) / *S;
  klen = std::max(SBK, (klen + SBK - 1) / SBK * SBK);
  *S = std::max(1, (K + klen - 1) / klen);   // planes actually written
  dim3 grid((M + SBM - 1) / SBM, (N + SBN - 1) / SBN, *S);
  skinny_partial_kernel<<<grid, 256, 0, s>>>(M, N, K, klen, A, lda, X, ldx, P, ldp, plane); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_gram_reduce(cudaStream_t s, const float* P, long long ldp, long long plane, int S, int mrows, int r,
                             int b, double* G, int n2) {
  dim3 grid((mrows + 255) / 256, b);
  gram_reduce_kernel<<<grid, 256, 0, s>>>(P, ldp, plane, S, mrows, r, b, G, n2); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_gram_rows_skinny(cudaStream_t s, const float* C, int ldc, int d, int r, int b, double* G, int n2,
                                  float* P, size_t p_cap) {
  const int M = r + b;
  int S = skinny_splits(M, b, d);
  while (S > 1 && (size_t)S * b * M > p_cap) --S;
  const long long ldp = M, plane = (long long)b * M;
  as_status st = launch_skinny_partial(s, M, b, d, &S, C, ldc, C + (long long)r * ldc, ldc, P, ldp, plane);
  if (st != AS_OK) return st;
  dim3 grid((M + 255) / 256, b);
  gram_reduce_kernel<<<grid, 256, 0, s>>>(P, ldp, plane, S, M, r, b, G, n2); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
