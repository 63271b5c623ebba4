// Block-speculative G-space iterations, the FP64 single-row path for large
// buffers, and the dump kernels.
//
// Within a block of b new rows and no event (no shrink, no dump), the buffer
// only grows by appending rows, so the state seen by row t of the block is the
// leading (r+t+1) x (r+t+1) principal submatrix of the block's Gram G.  The
// power iteration of every row (Algorithm 1) and the first doubling step
// (k = 2) of the simultaneous iteration of every row (Algorithm 2) are then
// independent problems on masked columns of one matrix:
//     X <- mask(G X)    (mask_t keeps rows < m_t = r + t + 1)
// and run as one split-K GEMM over G per iteration, followed by a per-row
// normalisation (k = 1) or SVQB orthonormalisation (k = 2).  These batched
// values locate the first row whose decision changes the state; that row is
// finished in FP64 (its Rayleigh-Ritz step reuses the batch's iterated basis)
// and rows whose batched value lies within a 1e-4 relative band of a
// threshold are re-decided by the FP64 power iteration.
//
// Batch matrix layout: column-major, column c at X + c*n2; columns [0, nb)
// are the power-iteration vectors of rows 0..nb-1 and columns nb+2t, nb+2t+1
// the simultaneous-iteration pair of row t.
#include <algorithm>

#include "eig.cuh"
#include "kernels.cuh"

namespace as {

namespace {

__global__ void batch_fill_kernel(float* X, int n2, int nb, int r0, Key key, uint64_t i0) {
  const int t = blockIdx.x, kind = blockIdx.y;  // kind 0: PI column, 1: SI pair
  const int m = r0 + t + 1;
  const uint64_t i = i0 + (uint64_t)t;
  if (kind == 0) {
    float* x = X + (size_t)t * n2;
    for (int blk = threadIdx.x; blk * 4 < n2; blk += blockDim.x) {
      double z[4];
      gauss4(key, kPurposePiStart, i, 0, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int p = blk * 4 + l;
        if (p < n2) x[p] = (p < m) ? (float)z[l] : 0.f;
      }
    }
  } else {
    float* x0 = X + (size_t)(nb + 2 * t) * n2;
    // Pi is n2 x 2 row-major: element e = 2p + c
    for (int blk = threadIdx.x; blk * 4 < 2 * n2; blk += blockDim.x) {
      double z[4];
      gauss4(key, kPurposeSiTest, i, 1, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int e = blk * 4 + l;
        if (e < 2 * n2) {
          const int p = e >> 1, c = e & 1;
          x0[(size_t)c * n2 + p] = (p < m) ? (float)z[l] : 0.f;
        }
      }
    }
  }
}

__device__ __forceinline__ void eig2(double s00, double s01, double s11, double& l0, double& l1, double& v00,
                                     double& v01, double& v10, double& v11) {
  const double tr = 0.5 * (s00 + s11), df = 0.5 * (s00 - s11);
  const double rad = sqrt(df * df + s01 * s01);
  l0 = tr + rad;
  l1 = tr - rad;
  if (rad == 0.0) { v00 = 1; v10 = 0; v01 = 0; v11 = 1; return; }
  const double th = 0.5 * atan2(2.0 * s01, s00 - s11);
  v00 = cos(th); v10 = sin(th); v01 = -v10; v11 = v00;
}

// After Y = G X (plane 0 of P after the split reduction): PI columns are
// normalised, SI pairs SVQB-orthonormalised (twice); on the final pass
// sigma^2 = x^T (G x) and the Ritz values of the pair are computed instead.
// Per-element arithmetic is FP32 (FP64 throughput is a small fraction of FP32
// on this part); only the per-thread partial sums are widened to FP64 for the
// block reductions and the 2 x 2 eigenproblems.  kind = kind0 + blockIdx.y.
__global__ void __launch_bounds__(512) batch_orth_kernel(const float* __restrict__ Y, float* X, int n2, int nb,
                                                         int r0, int kind0, int final_pi, int final_si,
                                                         double* sig2, double* ritz) {
  __shared__ double red[32];
  const int t = blockIdx.x, kind = kind0 + blockIdx.y;
  const int m = r0 + t + 1;
  if (kind == 0) {
    float* x = X + (size_t)t * n2;
    const float* y = Y + (size_t)t * n2;
    float sf = 0.f;
    if (final_pi) {
      for (int p = threadIdx.x; p < m; p += blockDim.x) sf = fmaf(x[p], y[p], sf);
      const double s = block_sum((double)sf, red);
      if (threadIdx.x == 0) sig2[t] = s;
      return;
    }
    for (int p = threadIdx.x; p < m; p += blockDim.x) sf = fmaf(y[p], y[p], sf);
    const double s = block_sum((double)sf, red);
    const float inv = (s > 0.0) ? (float)(1.0 / sqrt(s)) : 0.f;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) x[p] = (p < m) ? y[p] * inv : 0.f;
    return;
  }
  const size_t o0 = (size_t)(nb + 2 * t) * n2, o1 = o0 + n2;
  float* x0 = X + o0;
  float* x1 = X + o1;
  const float* y0 = Y + o0;
  const float* y1 = Y + o1;
  if (final_si) {
    // S = X^T (G X) (X orthonormal); SVQB -> W = X V D^-1/2, GW = Y V D^-1/2;
    // Ritz values = eig((GW)^T (GW)) = eig(D^-1/2 V^T (Y^T Y) V D^-1/2)
    float f00 = 0.f, f01 = 0.f, f11 = 0.f, g00 = 0.f, g01 = 0.f, g11 = 0.f;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const float a = x0[p], b = x1[p], ya = y0[p], yb = y1[p];
      f00 = fmaf(a, ya, f00); f01 = fmaf(0.5f, fmaf(a, yb, b * ya), f01); f11 = fmaf(b, yb, f11);
      g00 = fmaf(ya, ya, g00); g01 = fmaf(ya, yb, g01); g11 = fmaf(yb, yb, g11);
    }
    const double s00 = block_sum((double)f00, red), s01 = block_sum((double)f01, red), s11 = block_sum((double)f11, red);
    const double h00 = block_sum((double)g00, red), h01 = block_sum((double)g01, red), h11 = block_sum((double)g11, red);
    if (threadIdx.x == 0) {
      double l0, l1, v00, v01, v10, v11;
      eig2(s00, s01, s11, l0, l1, v00, v01, v10, v11);
      const double tol = 1e-6 * fmax(l0, 0.0);
      const double a0 = (l0 > tol && l0 > 0) ? 1.0 / sqrt(l0) : 0.0;
      const double a1 = (l1 > tol && l1 > 0) ? 1.0 / sqrt(l1) : 0.0;
      // M = diag(a) V^T H V diag(a), H = Y^T Y
      const double hv00 = h00 * v00 + h01 * v10, hv10 = h01 * v00 + h11 * v10;
      const double hv01 = h00 * v01 + h01 * v11, hv11 = h01 * v01 + h11 * v11;
      const double m00 = a0 * a0 * (v00 * hv00 + v10 * hv10);
      const double m01 = a0 * a1 * (v00 * hv01 + v10 * hv11);
      const double m11 = a1 * a1 * (v01 * hv01 + v11 * hv11);
      const double tr = 0.5 * (m00 + m11), df = 0.5 * (m00 - m11);
      const double rad = sqrt(df * df + m01 * m01);
      ritz[2 * t] = (a0 > 0) ? tr + rad : 0.0;
      ritz[2 * t + 1] = (a0 > 0 && a1 > 0) ? tr - rad : 0.0;
    }
    return;
  }
  // Euclidean SVQB of the pair: pass 0 reads Y, pass 1 re-orthonormalises X.
  // The 2 x 2 eigenproblem is solved once (thread 0, FP64) and broadcast.
  __shared__ float coef[4];
  for (int pass = 0; pass < 2; ++pass) {
    const float* s0 = pass ? x0 : y0;
    const float* s1 = pass ? x1 : y1;
    float f00 = 0.f, f01 = 0.f, f11 = 0.f;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const float a = s0[p], b = s1[p];
      f00 = fmaf(a, a, f00); f01 = fmaf(a, b, f01); f11 = fmaf(b, b, f11);
    }
    const double s00 = block_sum((double)f00, red), s01 = block_sum((double)f01, red), s11 = block_sum((double)f11, red);
    if (threadIdx.x == 0) {
      double l0, l1, v00, v01, v10, v11;
      eig2(s00, s01, s11, l0, l1, v00, v01, v10, v11);
      const double tol = 1e-13 * fmax(l0, 0.0);
      const double a0 = (l0 > tol && l0 > 0) ? 1.0 / sqrt(l0) : 0.0;
      const double a1 = (l1 > tol && l1 > 0) ? 1.0 / sqrt(l1) : 0.0;
      coef[0] = (float)(v00 * a0); coef[1] = (float)(v10 * a0);
      coef[2] = (float)(v01 * a1); coef[3] = (float)(v11 * a1);
    }
    __syncthreads();
    const float c00 = coef[0], c10 = coef[1], c01 = coef[2], c11 = coef[3];
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      float o0v = 0.f, o1v = 0.f;
      if (p < m) {
        const float a = s0[p], b = s1[p];
        o0v = fmaf(a, c00, b * c10);
        o1v = fmaf(a, c01, b * c11);
      }
      x0[p] = o0v;
      x1[p] = o1v;
    }
    __syncthreads();
  }
}

// Y(p, c) = sum_s P[s](p, c) for columns [c0, c1), rows < mmax, written into plane 0.
__global__ void plane_reduce_kernel(float* P, long long plane, int S, int n2, int c0, int c1, int mmax) {
  const int c = c0 + blockIdx.y;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < mmax; p += gridDim.x * blockDim.x) {
    const size_t off = (size_t)c * n2 + p;
    float v = 0.f;
    for (int s = 0; s < S; ++s) v += P[(long long)s * plane + off];
    P[off] = v;
  }
}

// Gf (FP32 mirror) = G (FP64) on the leading m x m block, zero elsewhere.
__global__ void mirror_f32_kernel(const double* G, float* Gf, int n2, int m) {
  const size_t tot = (size_t)n2 * n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / n2), q = (int)(e % n2);
    Gf[e] = (p < m && q < m) ? (float)G[e] : 0.f;
  }
}

__global__ void mirror_bf16_kernel(const double* G, int n2, int m, __nv_bfloat16* hi, __nv_bfloat16* lo, int n2p) {
  const size_t tot = (size_t)n2p * n2p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / n2p), q = (int)(e % n2p);
    const float x = (p < m && q < m) ? (float)G[(size_t)p * n2 + q] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

// ---- FP64 single-row path (any buffer size) ---------------------------------
__global__ void fill_pi_start(double* x, int n2, int m, Key key, uint64_t i) {
  for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < n2; blk += gridDim.x * blockDim.x) {
    double z[4];
    gauss4(key, kPurposePiStart, i, 0, blk, z);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int p = blk * 4 + l;
      if (p < n2) x[p] = (p < m) ? z[l] : 0.0;
    }
  }
}

__global__ void fill_si_test(double* Y, int n2, int m, int k, Key key, uint64_t i, int j) {
  const int tot = n2 * k;
  for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < tot; blk += gridDim.x * blockDim.x) {
    double z[4];
    gauss4(key, kPurposeSiTest, i, (uint64_t)j, blk, z);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = blk * 4 + l;
      if (e < tot) Y[e] = (e / k < m) ? z[l] : 0.0;
    }
  }
}

// Y[p][c] = sum_{q<m} G[p][q] X[q][c] for p < m, c < k <= KT (X, Y row-major n2 x k); one warp per row.
template <int KT>
__global__ void __launch_bounds__(256) gmul_thin_kernel(const double* __restrict__ G, int n2, int m, int k,
                                                       const double* __restrict__ X, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= m) return;
  const double* g = G + (size_t)p * n2;
  double acc[KT];
#pragma unroll
  for (int c = 0; c < KT; ++c) acc[c] = 0.0;
  for (int q = lane; q < m; q += 32) {
    const double gv = g[q];
#pragma unroll
    for (int c = 0; c < KT; ++c)
      if (c < k) acc[c] += gv * X[(size_t)q * k + c];
  }
#pragma unroll
  for (int c = 0; c < KT; ++c) {
    const double v = warp_sum(acc[c]);
    if (lane == 0 && c < k) Y[(size_t)p * k + c] = v;
  }
}

// x <- y / ||y|| (first m entries); *zero = 1 if ||y|| == 0.  One block.
__global__ void normalize_kernel(const double* y, double* x, int m, int* zero) {
  __shared__ double red[32];
  double s = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) s += y[p] * y[p];
  s = block_sum(s, red);
  if (s == 0.0) { if (threadIdx.x == 0) *zero = 1; return; }
  const double inv = 1.0 / sqrt(s);
  for (int p = threadIdx.x; p < m; p += blockDim.x) x[p] = y[p] * inv;
}

__global__ void dot_kernel(const double* x, const double* y, int m, const int* zero, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) s += x[p] * y[p];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = (*zero) ? 0.0 : s;
}

// S = sym(A^T B) over the first m rows (A, B row-major n2 x k).
__device__ void block_gram(int m, int k, const double* A, const double* B, double* S, double* red) {
  if (k <= 8) {
    for (int a = 0; a < k; ++a)
      for (int c = a; c < k; ++c) {
        double acc = 0.0;
        for (int p = threadIdx.x; p < m; p += blockDim.x)
          acc += 0.5 * (A[(size_t)p * k + a] * B[(size_t)p * k + c] + A[(size_t)p * k + c] * B[(size_t)p * k + a]);
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) { S[a * k + c] = acc; S[c * k + a] = acc; }
      }
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double acc = 0.0;
    for (int p = 0; p < m; ++p) acc += A[(size_t)p * k + a] * B[(size_t)p * k + c];
    S[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    if (a < c) { const double v = 0.5 * (S[a * k + c] + S[c * k + a]); S[a * k + c] = v; S[c * k + a] = v; }
  }
  __syncthreads();
}

// One block: SVQB of X with S = X^T X (or X^T Xg for the G inner product);
// X, Xg <- (.) V D^-1/2 on the kept columns.  Rows >= m are zero.
__global__ void svqb_kernel(int n2, int m, int k, double* X, double* Xg, int g_inner, double* S, double* V,
                            double* D, double* eigw, double* tmp) {
  __shared__ double red[32];
  block_gram(m, k, X, g_inner ? Xg : X, S, red);
  EigWork w = eig_work_view(eigw, k, k);
  cta_eig_sym(k, S, k, k, D, V, k, w, red);
  __syncthreads();
  const double dmax = D[0];
  const int passes = Xg ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    double* M = (pass == 0) ? X : Xg;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      for (int c = 0; c < k; ++c) {
        double acc = 0.0;
        if (p < m && dmax > 0.0 && D[c] > 1e-13 * dmax) {
          for (int a = 0; a < k; ++a) acc += M[(size_t)p * k + a] * V[a * k + c];
          acc /= sqrt(D[c]);
        }
        tmp[(size_t)p * k + c] = acc;
      }
      for (int c = 0; c < k; ++c) M[(size_t)p * k + c] = tmp[(size_t)p * k + c];
    }
    __syncthreads();
  }
}

// One block: with W G-orthonormal and GW: M = GW^T GW, eig -> ritz (descending), WU, GWU.
__global__ void rayleigh_ritz_kernel(int n2, int m, int k, const double* W, const double* GW, double* M, double* U,
                                     double* ritz, double* eigw, double* WU, double* GWU, int* status) {
  __shared__ double red[32];
  block_gram(m, k, GW, GW, M, red);
  EigWork w = eig_work_view(eigw, k, k);
  cta_eig_sym(k, M, k, k, ritz, U, k, w, red);
  __syncthreads();
  for (int e = threadIdx.x; e < n2 * k; e += blockDim.x) {
    const int p = e / k, c = e - p * k;
    double a1 = 0.0, a2 = 0.0;
    for (int a = 0; a < k; ++a) {
      a1 += W[(size_t)p * k + a] * U[a * k + c];
      a2 += GW[(size_t)p * k + a] * U[a * k + c];
    }
    WU[e] = a1;
    GWU[e] = a2;
  }
  if (threadIdx.x == 0 && !(ritz[0] == ritz[0])) set_status(status, AS_ENUMERIC);
}

// Rayleigh-Ritz of Algorithm 2 for k = 2 in FP64, one block, closed-form 2 x 2
// eigenproblems: S = Y^T (G Y) = V D V^T, W = Y V D^-1/2, GW = (G Y) V D^-1/2,
// M = GW^T GW = U diag(ritz) U^T, WU, GWU.  Y is orthonormal (Euclidean).
__global__ void rr2_kernel(int n2, int m, const double* Y, const double* GY, double* ritz, double* WU, double* GWU,
                           int* status) {
  __shared__ double red[32];
  __shared__ double cf[8];   // (v00, v10, v01, v11) * (a0, a0, a1, a1), then U
  double s00 = 0, s01 = 0, s11 = 0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const double a = Y[2 * p], b = Y[2 * p + 1], ga = GY[2 * p], gb = GY[2 * p + 1];
    s00 += a * ga; s01 += 0.5 * (a * gb + b * ga); s11 += b * gb;
  }
  s00 = block_sum(s00, red); s01 = block_sum(s01, red); s11 = block_sum(s11, red);
  if (threadIdx.x == 0) {
    double l0, l1, v00, v01, v10, v11;
    eig2(s00, s01, s11, l0, l1, v00, v01, v10, v11);
    const double a0 = (l0 > 0.0) ? 1.0 / sqrt(l0) : 0.0;
    const double a1 = (l1 > 1e-13 * l0 && l1 > 0.0) ? 1.0 / sqrt(l1) : 0.0;
    cf[0] = v00 * a0; cf[1] = v10 * a0; cf[2] = v01 * a1; cf[3] = v11 * a1;
  }
  __syncthreads();
  const double w00 = cf[0], w10 = cf[1], w01 = cf[2], w11 = cf[3];
  // G W columns
  double m00 = 0, m01 = 0, m11 = 0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    const double ga = GY[2 * p], gb = GY[2 * p + 1];
    const double g0 = ga * w00 + gb * w10, g1 = ga * w01 + gb * w11;
    m00 += g0 * g0; m01 += g0 * g1; m11 += g1 * g1;
  }
  m00 = block_sum(m00, red); m01 = block_sum(m01, red); m11 = block_sum(m11, red);
  if (threadIdx.x == 0) {
    double r0, r1, u00, u01, u10, u11;
    eig2(m00, m01, m11, r0, r1, u00, u01, u10, u11);
    ritz[0] = r0;
    ritz[1] = (w01 != 0.0 || w11 != 0.0) ? r1 : 0.0;
    if (!(r0 == r0)) set_status(status, AS_ENUMERIC);
    cf[4] = u00; cf[5] = u10; cf[6] = u01; cf[7] = u11;
  }
  __syncthreads();
  const double u00 = cf[4], u10 = cf[5], u01 = cf[6], u11 = cf[7];
  for (int p = threadIdx.x; p < n2; p += blockDim.x) {
    double w0 = 0, w1 = 0, g0 = 0, g1 = 0;
    if (p < m) {
      const double a = Y[2 * p], b = Y[2 * p + 1], ga = GY[2 * p], gb = GY[2 * p + 1];
      const double x0 = a * w00 + b * w10, x1 = a * w01 + b * w11;      // W
      const double y0 = ga * w00 + gb * w10, y1 = ga * w01 + gb * w11;  // G W
      w0 = x0 * u00 + x1 * u10; w1 = x0 * u01 + x1 * u11;
      g0 = y0 * u00 + y1 * u10; g1 = y0 * u01 + y1 * u11;
    }
    WU[2 * p] = w0; WU[2 * p + 1] = w1;
    GWU[2 * p] = g0; GWU[2 * p + 1] = g1;
  }
}

__global__ void promote_pair_kernel(const float* X, int n2, int col0, int m, int k, double* Y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * k; e += gridDim.x * blockDim.x) {
    const int p = e / k, c = e - p * k;
    Y[e] = (p < m) ? (double)X[(size_t)(col0 + c) * n2 + p] : 0.0;
  }
}

// ---- dump (Algorithm 4 lines 14-16) -----------------------------------------
// Partial sums over row chunks s: Zp[s][c][a] = sum_p C[p][c] WU[p][a] and
// Yp[s][a][c] = sum_p GWU[p][a] C[p][c] for a in [a0, a0+na), one thread per column c.
constexpr int kDumpChunks = 8;
__global__ void dump_partial_kernel(const float* __restrict__ C, int ldc, int d, int r, const double* WU,
                                    const double* GWU, int k, int xi, int a0, int na, double* Zp, double* Yp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (c >= d) return;
  const int chunk = (r + kDumpChunks - 1) / kDumpChunks;
  const int pb = s * chunk, pe = min(r, pb + chunk);
  double z[8], y[8];
  float zf[8], yf[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) { z[a] = 0.0; y[a] = 0.0; zf[a] = 0.f; yf[a] = 0.f; }
  int cnt = 0;
  for (int p = pb; p < pe; ++p) {
    const float cv = C[(size_t)p * ldc + c];
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (a < na) {
        zf[a] = fmaf(cv, (float)WU[(size_t)p * k + a0 + a], zf[a]);
        yf[a] = fmaf(cv, (float)GWU[(size_t)p * k + a0 + a], yf[a]);
      }
    if (++cnt == 64) {   // FP32 partial sums of 64 rows, combined in FP64
      cnt = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) { z[a] += zf[a]; y[a] += yf[a]; zf[a] = 0.f; yf[a] = 0.f; }
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a)
    if (a < na) {
      Zp[((size_t)s * d + c) * xi + a0 + a] = z[a] + zf[a];
      Yp[((size_t)s * xi + a0 + a) * d + c] = y[a] + yf[a];
    }
}

__global__ void dump_reduce_kernel(const double* Zp, const double* Yp, int d, int xi, float* Z, float* Y) {
  const int tot = d * xi;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    double z = 0.0, y = 0.0;
    for (int s = 0; s < kDumpChunks; ++s) { z += Zp[(size_t)s * tot + e]; y += Yp[(size_t)s * tot + e]; }
    Z[e] = (float)z;   // Z: d x xi row-major (e = c*xi + a)
    Y[e] = (float)y;   // Y: xi x d row-major (e = a*d + c)
  }
}

// C[p][c] -= sum_a GWU[p][a] Z[c][a]   (the residual C' - C' Z Z^T)
__global__ void residual_kernel(float* C, int ldc, int d, int r, const double* GWU, int k, int xi, const float* Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (c >= d || p >= r) return;
  double acc = 0.0;
  for (int a = 0; a < xi; ++a) acc += GWU[(size_t)p * k + a] * (double)Z[(size_t)c * xi + a];
  C[(size_t)p * ldc + c] = (float)((double)C[(size_t)p * ldc + c] - acc);
}

// G[p][q] -= sum_a GWU[p][a] GWU[q][a]
__global__ void gram_downdate_kernel(double* G, int n2, int r, const double* GWU, int k, int xi) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (q >= r || p >= r) return;
  double acc = 0.0;
  for (int a = 0; a < xi; ++a) acc += GWU[(size_t)p * k + a] * GWU[(size_t)q * k + a];
  G[(size_t)p * n2 + q] -= acc;
}

}  // namespace

as_status launch_gf_mirror(cudaStream_t s, const double* G, float* Gf, int n2, int m) {
  const size_t tot = (size_t)n2 * n2;
  const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
  mirror_f32_kernel<<<blocks, 256, 0, s>>>(G, Gf, n2, m); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_gbf16_mirror(cudaStream_t s, const double* G, int n2, int m, __nv_bfloat16* hi, __nv_bfloat16* lo,
                              int n2p) {
  const size_t tot = (size_t)n2p * n2p;
  const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
  mirror_bf16_kernel<<<blocks, 256, 0, s>>>(G, n2, m, hi, lo, n2p); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_batch_gspace(cudaStream_t s, const float* Gf, int n2, int r0, int nb, int k_pi, int q, Key key,
                              uint64_t i0, const BatchBuffers& bb, Prof* prof, const TcBatch* tc) {
  if (nb <= 0) return AS_OK;
  const int ncol = 3 * nb;
  const int mmax = r0 + nb;
  const long long plane = (long long)n2 * ncol;
  batch_fill_kernel<<<dim3(nb, 2), 128, 0, s>>>(bb.X, n2, nb, r0, key, i0); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  if (tc) {
    as_status st = launch_split_bf16(s, bb.X, n2, ncol, n2, tc->Xh, tc->Xl, tc->n2p, false);
    if (st != AS_OK) return st;
  }
  const int iters = std::max(k_pi, q);
  for (int it = 0; it <= iters; ++it) {
    const bool pi_on = it <= k_pi;
    const bool si_on = it <= q;
    const int c0 = pi_on ? 0 : nb;
    const int c1 = si_on ? ncol : nb;
    int S = std::min(skinny_splits(mmax, c1 - c0, mmax), bb.max_splits);
    if (prof) prof->begin(PK_BATCH_GEMM, s);
    as_status st;
    if (tc) {
      // split-BF16 tcgen05 product Y = G X: A = G (rows p, K = q), B = X^T (rows c, K = q)
      const int Kp = (mmax + 63) / 64 * 64;
      const int ktiles = Kp / 64;
      const int mt = (mmax + 127) / 128;
      S = std::max(1, std::min({(2 * 152 + mt - 1) / mt, ktiles, bb.max_splits}));
      const int klen = ((ktiles + S - 1) / S) * 64;
      S = (Kp + klen - 1) / klen;
      st = launch_umma_gemm(s, *tc->mapG, *tc->mapX, mmax, c1 - c0, Kp, 192,
                            3, S, c0, bb.P + (size_t)c0 * n2, 1, n2, plane, tc->err);
    } else {
      st = launch_skinny_partial(s, mmax, c1 - c0, mmax, &S, Gf, n2, bb.X + (size_t)c0 * n2, n2,
                                 bb.P + (size_t)c0 * n2, n2, plane);
    }
    if (st != AS_OK) return st;
    // algorithmic work of one product: 2 m^2 N flops; G (m^2 FP32) and X read, Y written
    if (prof)
      prof->end(PK_BATCH_GEMM, s, 2.0 * mmax * (double)mmax * (c1 - c0),
                4.0 * ((double)mmax * mmax + 2.0 * (double)mmax * (c1 - c0)));
    if (prof) prof->begin(PK_BATCH_ORTH, s);
    if (S > 1) {
      plane_reduce_kernel<<<dim3((mmax + 255) / 256, c1 - c0), 256, 0, s>>>(bb.P, plane, S, n2, c0, c1, mmax); count_launches(1);
    }
    // PI: iterations 0..k_pi-1 normalise, k_pi evaluates sigma^2;
    // SI: iterations 0..q-1 orthonormalise, q does Rayleigh-Ritz.
    const int kind0 = pi_on ? 0 : 1;
    const int kinds = (pi_on ? 1 : 0) + (si_on ? 1 : 0);
    batch_orth_kernel<<<dim3(nb, kinds), 512, 0, s>>>(bb.P, bb.X, n2, nb, r0, kind0, it == k_pi ? 1 : 0,
                                                      it == q ? 1 : 0, bb.sig2, bb.ritz); count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
    if (tc && it < iters) {
      const int nc0 = (it + 1 <= k_pi) ? 0 : nb;   // columns the next product reads
      st = launch_split_bf16(s, bb.X + (size_t)nc0 * n2, n2, ncol - nc0, n2, tc->Xh + (size_t)nc0 * tc->n2p,
                             tc->Xl + (size_t)nc0 * tc->n2p, tc->n2p, false);
      if (st != AS_OK) return st;
    }
    if (prof) prof->end(PK_BATCH_ORTH, s, 0.0, 4.0 * (double)mmax * (c1 - c0) * (S + 2));
  }
  return AS_OK;
}

static as_status gmul_thin(cudaStream_t s, const double* G, int n2, int m, int k, const double* X, double* Y) {
  const int grid = (m + 7) / 8;
  if (k <= 2) {
    gmul_thin_kernel<2><<<grid, 256, 0, s>>>(G, n2, m, k, X, Y); count_launches(1);
  } else {
    gmul_thin_kernel<8><<<grid, 256, 0, s>>>(G, n2, m, k, X, Y); count_launches(1);
  }
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

// products by G for the FP64 single-row path: thin kernel for k <= 8, else the tiled GEMM
static as_status gmul64(cudaStream_t s, const double* G, int n2, int m, int k, const double* X, double* Y) {
  if (k <= 8) return gmul_thin(s, G, n2, m, k, X, Y);
  return gemm_strided<double, double, double>(s, m, k, m, G, n2, 1, X, k, 1, Y, k, 1, 1.0, 0.0);
}

as_status launch_power_iteration_f64(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key, uint64_t i,
                                     double* x, double* y, int* zero, double* sig2) {
  AS_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(int), s));
  fill_pi_start<<<(n2 / 4 + 255) / 256 + 1, 256, 0, s>>>(x, n2, m, key, i); count_launches(1);
  normalize_kernel<<<1, 512, 0, s>>>(x, x, m, zero); count_launches(1);
  for (int it = 0; it < k_pi; ++it) {
    as_status st = gmul64(s, G, n2, m, 1, x, y);
    if (st != AS_OK) return st;
    normalize_kernel<<<1, 512, 0, s>>>(y, x, m, zero); count_launches(1);
  }
  as_status st = gmul64(s, G, n2, m, 1, x, y);
  if (st != AS_OK) return st;
  dot_kernel<<<1, 512, 0, s>>>(x, y, m, zero, sig2); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_simul_iter_f64(cudaStream_t s, const double* G, int n2, int m, int k, int q, Key key, uint64_t i,
                                int j, const SiBuffers& b, int* status) {
  fill_si_test<<<((n2 * k) / 4 + 255) / 256 + 1, 256, 0, s>>>(b.Y, n2, m, k, key, i, j); count_launches(1);
  AS_CUDA_TRY(cudaMemsetAsync(b.GY, 0, (size_t)n2 * k * sizeof(double), s));
  for (int t = 0; t < q; ++t) {
    as_status st = gmul64(s, G, n2, m, k, b.Y, b.GY);
    if (st != AS_OK) return st;
    for (int pass = 0; pass < 2; ++pass) {
      svqb_kernel<<<1, 512, 0, s>>>(n2, m, k, b.GY, nullptr, 0, b.S, b.V, b.ritz, b.eigw, b.tmp); count_launches(1);
    }
    AS_CUDA_TRY(cudaMemcpyAsync(b.Y, b.GY, (size_t)n2 * k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  as_status st = gmul64(s, G, n2, m, k, b.Y, b.GY);
  if (st != AS_OK) return st;
  svqb_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, 1, b.S, b.V, b.ritz, b.eigw, b.tmp); count_launches(1);
  rayleigh_ritz_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, b.S, b.V, b.ritz, b.eigw, b.WU, b.GWU, status); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_si_rr_from_batch(cudaStream_t s, const double* G, int n2, int m, const float* X, int col0,
                                  const SiBuffers& b, int* status) {
  const int k = 2;
  promote_pair_kernel<<<(n2 * k + 255) / 256, 256, 0, s>>>(X, n2, col0, m, k, b.Y); count_launches(1);
  AS_CUDA_TRY(cudaMemsetAsync(b.GY, 0, (size_t)n2 * k * sizeof(double), s));
  as_status st = gmul64(s, G, n2, m, k, b.Y, b.GY);
  if (st != AS_OK) return st;
  rr2_kernel<<<1, 1024, 0, s>>>(n2, m, b.Y, b.GY, b.ritz, b.WU, b.GWU, status); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

size_t dump_work_doubles(int d, int xi) { return (size_t)2 * kDumpChunks * d * xi; }

as_status launch_dump(cudaStream_t s, float* C, int ldc, int d, int r, double* G, int n2, const double* WU,
                      const double* GWU, int k, int xi, float* Z, float* Y, double* work) {
  double* Zp = work;
  double* Yp = work + (size_t)kDumpChunks * d * xi;
  for (int a0 = 0; a0 < xi; a0 += 8) {
    const int na = std::min(8, xi - a0);
    dim3 grid((d + 127) / 128, kDumpChunks);
    dump_partial_kernel<<<grid, 128, 0, s>>>(C, ldc, d, r, WU, GWU, k, xi, a0, na, Zp, Yp); count_launches(1);
  }
  dump_reduce_kernel<<<(d * xi + 255) / 256, 256, 0, s>>>(Zp, Yp, d, xi, Z, Y); count_launches(1);
  if (r > 0) {
    residual_kernel<<<dim3((d + 255) / 256, r), 256, 0, s>>>(C, ldc, d, r, GWU, k, xi, Z); count_launches(1);
    gram_downdate_kernel<<<dim3((r + 255) / 256, r), 256, 0, s>>>(G, n2, r, GWU, k, xi); count_launches(1);
  }
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
