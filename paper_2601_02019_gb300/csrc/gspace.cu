// Row ingest, Gram maintenance and the G-space iterations of AeroSketch.
//
// The buffer C (2l x d) enters the power iteration and the simultaneous
// iteration only through products with C' C'^T (Algorithm 1 with A = C'^T
// multiplies by A^T A = C' C'^T) and with C'^T C' (Algorithm 2).  Keeping the
// 2l x 2l Gram G = C C^T lets both run in the 2l-dimensional row space:
//   power iteration   x <- G x / ||G x||,  sigma^2 = x^T G x;
//   simultaneous it.  K = C'^T Y with Y = G^q Pi, so the span is iterated as
//                     Y <- orth(G Y), and the Rayleigh-Ritz step uses
//                     S = Y^T G Y (the Gram of K) and M = W^T G^2 W for a
//                     G-orthonormal W (so that Q = C'^T W is orthonormal).
#include "eig.cuh"
#include "kernels.cuh"

namespace as {

namespace {

// ----------------------------------------------------------------- ingest --
__global__ void ingest_kernel(const float* __restrict__ rows, long long ld_in, int n, int d,
                              float* __restrict__ C, int ldc, int r, double* norm2, int* bad) {
  const int t = blockIdx.x;
  if (t >= n) return;
  const float* src = rows + (long long)t * ld_in;
  float* dst = C + (long long)(r + t) * ldc;
  double s = 0.0;
  int nonfinite = 0;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    const float v = src[c];
    const bool ok = isfinite(v);
    nonfinite |= !ok;
    dst[c] = ok ? v : 0.f;   // a rejected row never reaches the products as NaN / Inf
    s += ok ? (double)v * (double)v : 0.0;
  }
  __shared__ double red[32];
  s = block_sum(s, red);
  nonfinite = __syncthreads_or(nonfinite);
  if (threadIdx.x == 0) {
    norm2[t] = nonfinite ? __longlong_as_double(0x7ff8000000000000ll) : s;   // NaN marks the row
    if (nonfinite) atomicExch(bad, 1);
  }
}

__global__ void truncate_kernel(float* C, int ldc, int d, int r0, int r1, double* G, int n2) {
  const long long tot_c = (long long)(r1 - r0) * ldc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_c;
       e += (long long)gridDim.x * blockDim.x)
    C[(long long)r0 * ldc + e] = 0.f;
  // G: rows [r0, r1) in full, then columns [r0, r1) of rows [0, r0).  Rows
  // and columns past r1 are zero already: a block writes G only up to its
  // last row r1, and every cut zeroes what the block wrote past the cut.
  const long long w = r1 - r0;
  const long long tot_g = w * n2 + (long long)r0 * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_g;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < w * n2) {
      G[(long long)r0 * n2 + e] = 0.0;
    } else {
      const long long f = e - w * n2;
      const long long p = f / w, q = r0 + f % w;
      G[p * n2 + q] = 0.0;
    }
  }
}

__global__ void mirror_kernel(double* G, int n2, int r, int b) {
  // copy G[p][r+t] (p < r) into G[r+t][p]
  const int t = blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < r; p += gridDim.x * blockDim.x)
    G[(long long)(r + t) * n2 + p] = G[(long long)p * n2 + r + t];
}

// ---------------------------------------------------------- power iteration --
// One block; x and y live in shared memory (2 * n2 doubles).
__global__ void power_iteration_kernel(const double* __restrict__ G, int n2, int m, int k_pi, Key key, uint64_t jsub,
                                       uint64_t i, double* sig2) {
  extern __shared__ double sm[];
  double* x = sm;
  double* y = sm + n2;
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  // x^(0) ~ N(0, I_{2l}) (Philox purpose 3, (i, jsub)); entries of empty rows do
  // not reach G x, so only the first m are kept (the normalisation of x^(0)
  // does not change the direction of G x^(0)).
  for (int blk = tid; blk * 4 < n2; blk += nt) {
    double z[4];
    gauss4(key, kPurposePiStart, i, jsub, blk, z);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = blk * 4 + l;
      if (e < n2) x[e] = (e < m) ? z[l] : 0.0;
    }
  }
  __syncthreads();
  double nrm2 = 0.0;
  for (int p = tid; p < m; p += nt) nrm2 += x[p] * x[p];
  nrm2 = block_sum(nrm2, red);
  if (nrm2 == 0.0) { if (tid == 0) *sig2 = 0.0; return; }
  const double inv0 = 1.0 / sqrt(nrm2);
  for (int p = tid; p < m; p += nt) x[p] *= inv0;
  __syncthreads();
  for (int it = 0; it < k_pi; ++it) {
    double part = 0.0;
    for (int p = tid; p < m; p += nt) {
      const double* g = G + (long long)p * n2;
      double acc = 0.0;
      for (int q = 0; q < m; ++q) acc += g[q] * x[q];
      y[p] = acc;
      part += acc * acc;
    }
    const double ny2 = block_sum(part, red);
    if (ny2 == 0.0) { if (tid == 0) *sig2 = 0.0; return; }
    const double inv = 1.0 / sqrt(ny2);
    for (int p = tid; p < m; p += nt) x[p] = y[p] * inv;
    __syncthreads();
  }
  double part = 0.0;
  for (int p = tid; p < m; p += nt) {
    const double* g = G + (long long)p * n2;
    double acc = 0.0;
    for (int q = 0; q < m; ++q) acc += g[q] * x[q];
    part += x[p] * acc;
  }
  const double s2 = block_sum(part, red);
  if (tid == 0) *sig2 = s2;
}

// ------------------------------------------------------ simultaneous iteration --
// Out[p][c] = sum_{q<m} G[p][q] In[q][c] for p < m; rows >= m are zero.
__device__ void cta_gmul(const double* G, int n2, int m, int k, const double* In, double* Out) {
  for (int e = threadIdx.x; e < n2 * k; e += blockDim.x) {
    const int p = e / k, c = e - p * k;
    double acc = 0.0;
    if (p < m) {
      const double* g = G + (long long)p * n2;
      for (int q = 0; q < m; ++q) acc += g[q] * In[q * k + c];
    }
    Out[e] = acc;
  }
  __syncthreads();
}

// S = A^T B for n2 x k matrices (rows < m).
__device__ void cta_gram(int m, int k, const double* A, const double* B, double* S) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, b = e - a * k;
    double acc = 0.0;
    for (int p = 0; p < m; ++p) acc += A[p * k + a] * B[p * k + b];
    S[e] = acc;
  }
  __syncthreads();
}

// SVQB orthonormalisation (Stathopoulos & Wu): with S = X^T B X = V D V^T,
// X <- X V D^{-1/2} (columns with D <= tol * max D set to zero), and the same
// right factor applied to Xg (the image of X under G, or nullptr).
// Returns the number of kept columns (kept columns come first).
__device__ int cta_svqb(int n2, int m, int k, double* X, double* Xg, double* S, double* V, double* D,
                        double* eigw, double* tmp, double* red) {
  EigWork w = eig_work_view(eigw, k, k);
  cta_eig_sym(k, S, k, k, D, V, k, w, red);
  __syncthreads();
  const double dmax = D[0];
  __shared__ int kept_s;
  if (threadIdx.x == 0) {
    int kept = 0;
    for (int c = 0; c < k; ++c)
      if (D[c] > 1e-13 * dmax && D[c] > 0.0) ++kept;
    kept_s = (dmax > 0.0) ? kept : 0;
  }
  __syncthreads();
  const int kept = kept_s;
  for (int pass = 0; pass < (Xg ? 2 : 1); ++pass) {
    double* M = (pass == 0) ? X : Xg;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      for (int c = 0; c < k; ++c) {
        double acc = 0.0;
        if (c < kept && p < m) {
          for (int a = 0; a < k; ++a) acc += M[p * k + a] * V[a * k + c];
          acc /= sqrt(D[c]);
        }
        tmp[p * k + c] = acc;
      }
      for (int c = 0; c < k; ++c) M[p * k + c] = tmp[p * k + c];
    }
    __syncthreads();
  }
  return kept;
}

__global__ void simul_iter_kernel(const double* __restrict__ G, int n2, int m, int k, int q, Key key,
                                  uint64_t i, int j, SiBuffers b, double* tmp, int* status) {
  __shared__ double red[32];
  double* Y = b.Y;
  double* GY = b.GY;
  // Pi ~ N(0,1)^{2l x k} (Philox purpose 4, (i, j)), row-major; rows of empty
  // buffer rows do not reach K = C'^T Pi and are dropped.
  const int tot = n2 * k;
  for (int blk = threadIdx.x; blk * 4 < tot; blk += blockDim.x) {
    double z[4];
    gauss4(key, kPurposeSiTest, i, (uint64_t)j, blk, z);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = blk * 4 + l;
      if (e < tot) Y[e] = (e / k < m) ? z[l] : 0.0;
    }
  }
  __syncthreads();
  // Y <- orth(G^t Pi), t = 1..q (Euclidean SVQB after every product)
  for (int t = 0; t < q; ++t) {
    cta_gmul(G, n2, m, k, Y, GY);
    for (int pass = 0; pass < 2; ++pass) {   // SVQB twice, as CholQR2 does
      cta_gram(m, k, GY, GY, b.S);
      cta_svqb(n2, m, k, GY, nullptr, b.S, b.V, b.ritz, b.eigw, tmp, red);
    }
    for (int e = threadIdx.x; e < tot; e += blockDim.x) Y[e] = GY[e];
    __syncthreads();
  }
  // Rayleigh-Ritz: W = G-orthonormal basis of span(Y) (S = Y^T G Y), then
  // M = (G W)^T (G W), eig(M) = U diag(sigma^2) U^T, outputs W U and G W U.
  cta_gmul(G, n2, m, k, Y, GY);
  cta_gram(m, k, Y, GY, b.S);
  const int kept = cta_svqb(n2, m, k, Y, GY, b.S, b.V, b.ritz, b.eigw, tmp, red);
  // Y = W (n2 x k, first `kept` columns), GY = G W
  cta_gram(m, k, GY, GY, b.S);
  // restrict the eigenproblem to the kept block (columns >= kept are zero)
  __shared__ int kk_s;
  if (threadIdx.x == 0) kk_s = kept;
  __syncthreads();
  const int kk = kk_s;
  if (kk == 0) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) b.ritz[c] = 0.0;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) { b.WU[e] = 0.0; b.GWU[e] = 0.0; }
    return;
  }
  // compact M (k x k with zero tail) into a kk x kk matrix in tmp
  double* M = tmp;
  for (int e = threadIdx.x; e < kk * kk; e += blockDim.x) {
    const int a = e / kk, c = e - a * kk;
    M[e] = 0.5 * (b.S[a * k + c] + b.S[c * k + a]);
  }
  __syncthreads();
  double* U = tmp + kk * kk;
  double* sig = tmp + 2 * kk * kk;
  EigWork w = eig_work_view(b.eigw, kk, kk);
  cta_eig_sym(kk, M, kk, kk, sig, U, kk, w, red);
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) b.ritz[c] = (c < kk) ? sig[c] : 0.0;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = e / k, c = e - p * k;
    double a1 = 0.0, a2 = 0.0;
    if (c < kk) {
      for (int a = 0; a < kk; ++a) {
        a1 += Y[p * k + a] * U[a * kk + c];
        a2 += GY[p * k + a] * U[a * kk + c];
      }
    }
    b.WU[e] = a1;
    b.GWU[e] = a2;
  }
  if (threadIdx.x == 0 && !(sig[0] == sig[0])) set_status(status, AS_ENUMERIC);
}

__global__ void eig_kernel(int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                           double* work) {
  __shared__ double red[32];
  EigWork w = eig_work_view(work, n, nev);
  cta_eig_sym(n, A, lda, nev, evals, X, ldx, w, red);
}

// Column j < l-1 of U: flip so that its largest-magnitude entry (lowest index
// on exact ties) is positive, then scale into W[j] (FP32).
__global__ void shrink_weights_kernel(int n2, int ell, const double* lam, double* U, float* W) {
  const int j = blockIdx.x;
  if (j >= ell - 1) return;
  __shared__ double bv[32];
  __shared__ int bi[32];
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int p = threadIdx.x; p < n2; p += blockDim.x) {
    const double a = fabs(U[(long long)p * ell + j]);
    if (a > best || (a == best && p < bidx)) { best = a; bidx = p; }
  }
  // block argmax (ties -> lowest index)
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > best || (bv[w] == best && bi[w] < bidx)) { best = bv[w]; bidx = bi[w]; }
    bi[0] = bidx;
  }
  __syncthreads();
  const double sgn = (U[(long long)bi[0] * ell + j] < 0.0) ? -1.0 : 1.0;
  const double lj = lam[j], ll = lam[ell - 1];
  const double sc = (lj > 0.0 && lj > ll) ? sqrt((lj - ll) / lj) : 0.0;
  for (int p = threadIdx.x; p < n2; p += blockDim.x) {
    const double u = sgn * U[(long long)p * ell + j];
    U[(long long)p * ell + j] = u;
    W[(long long)j * n2 + p] = (float)(sc * u);
  }
}

__global__ void shrink_rows_kernel(int d, int ell, const double* lam, const double* V, int ldv, float* out,
                                   long long ldo) {
  const int j = blockIdx.x;
  const double sc = sqrt(fmax(lam[j] - lam[ell - 1], 0.0));
  for (int c = threadIdx.x; c < d; c += blockDim.x) out[(long long)j * ldo + c] = (float)(sc * V[(long long)c * ldv + j]);
}

}  // namespace

as_status launch_ingest(cudaStream_t s, const float* rows, long long ld_in, int n, int d, float* C, int ldc,
                        int r, double* norm2, int* bad) {
  if (n <= 0) return AS_OK;
  ingest_kernel<<<n, 256, 0, s>>>(rows, ld_in, n, d, C, ldc, r, norm2, bad); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_truncate(cudaStream_t s, float* C, int ldc, int d, int r0, int r1, double* G, int n2) {
  truncate_kernel<<<128, 256, 0, s>>>(C, ldc, d, r0, r1, G, n2); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_gram_rows(cudaStream_t s, const float* C, int ldc, int d, int r, int b, double* G, int n2) {
  // G[p][r+t] = sum_c C[p][c] C[r+t][c], p < r+b
  as_status st = gemm_strided<float, float, double>(s, r + b, b, d, C, ldc, 1, C + (long long)r * ldc, 1, ldc,
                                                    G + r, n2, 1, 1.0, 0.0);
  if (st != AS_OK) return st;
  if (r > 0) {
    dim3 grid((r + 255) / 256, b);
    mirror_kernel<<<grid, 256, 0, s>>>(G, n2, r, b); count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
  }
  return AS_OK;
}

as_status launch_power_iteration(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key, uint64_t i,
                                 double* sig2, uint64_t jsub) {
  const size_t smem = 2 * (size_t)n2 * sizeof(double);
  AS_CUDA_TRY(as_raise_smem_limit((const void*)power_iteration_kernel, smem));
  power_iteration_kernel<<<1, 512, smem, s>>>(G, n2, m, k_pi, key, jsub, i, sig2); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_simul_iter(cudaStream_t s, const double* G, int n2, int m, int k, int q, Key key, uint64_t i,
                            int j, const SiBuffers& b, int* status) {
  simul_iter_kernel<<<1, 512, 0, s>>>(G, n2, m, k, q, key, i, j, b, b.tmp, status); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_eig(cudaStream_t s, int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                     double* work) {
  eig_kernel<<<1, 512, 0, s>>>(n, A, lda, nev, evals, X, ldx, work); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_shrink_weights(cudaStream_t s, int n2, int ell, const double* lam, double* U, float* W) {
  if (ell <= 1) return AS_OK;
  shrink_weights_kernel<<<ell - 1, 256, 0, s>>>(n2, ell, lam, U, W); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_shrink_rows(cudaStream_t s, int d, int ell, const double* lam, const double* V, int ldv,
                             float* out, long long ldo) {
  shrink_rows_kernel<<<ell, 256, 0, s>>>(d, ell, lam, V, ldv, out, ldo); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
