// Block-speculative G-space iterations and the FP64 single-row path for large buffers.
//
// Within a block of b new rows and no event (no shrink, no dump), the buffer
// only grows by appending rows, so the state seen by row t of the block is the
// leading (r+t+1) x (r+t+1) principal submatrix of the block's Gram G.  The
// power iteration of every row (Algorithm 1) and the first doubling step
// (k = 2) of the simultaneous iteration of every row (Algorithm 2) are then
// independent problems on masked columns of one matrix:
//     X <- mask(G X)    (mask_t keeps rows < m_t = r + t + 1)
// and run as one GEMM over G per iteration, followed by a per-row
// normalisation (k = 1) or SVQB orthonormalisation (k = 2).  These batched
// values are only used to locate the first row whose decision changes the
// state; that row, and any row whose batched value lies within a 1e-4
// relative band of a threshold, is recomputed by the FP64 single-row path.
#include "eig.cuh"
#include "kernels.cuh"

namespace as {

namespace {

// Column layout of the batch matrix X (n2 x ncol, row-major, ld = ncol):
//   columns [0, nb)          : power-iteration vectors of rows 0..nb-1
//   columns [nb + 2t, +2)    : simultaneous-iteration pair of row t
__global__ void batch_fill_kernel(float* X, int n2, int ncol, int nb, int r0, Key key, uint64_t i0) {
  // one block per (row t, kind); kind 0 = PI column, kind 1 = SI pair
  const int t = blockIdx.x, kind = blockIdx.y;
  const int m = r0 + t + 1;
  const uint64_t i = i0 + (uint64_t)t;
  if (kind == 0) {
    for (int blk = threadIdx.x; blk * 4 < n2; blk += blockDim.x) {
      double z[4];
      gauss4(key, kPurposePiStart, i, 0, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int p = blk * 4 + l;
        if (p < n2) X[(size_t)p * ncol + t] = (p < m) ? (float)z[l] : 0.f;
      }
    }
  } else {
    // Pi is n2 x 2 row-major: element e = 2p + c
    for (int blk = threadIdx.x; blk * 4 < 2 * n2; blk += blockDim.x) {
      double z[4];
      gauss4(key, kPurposeSiTest, i, 1, blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int e = blk * 4 + l;
        if (e < 2 * n2) {
          const int p = e >> 1, c = e & 1;
          X[(size_t)p * ncol + nb + 2 * t + c] = (p < m) ? (float)z[l] : 0.f;
        }
      }
    }
  }
}

// After Y = G X: mask rows >= m_t and normalise (PI) or SVQB-orthonormalise
// (SI pair) each problem's columns; the result goes back into X.
// On the final pass (final = 1) instead compute sigma^2 (PI: x^T G x with
// X = x, Y = G x) and the two Ritz values (SI: S = X^T Y, M = (GW)^T(GW)).
__global__ void batch_orth_kernel(const float* Y, float* X, int n2, int ncol, int nb, int r0, int pi_active,
                                  int final, double* sig2, double* ritz) {
  __shared__ double red[32];
  const int t = blockIdx.x, kind = blockIdx.y;
  const int m = r0 + t + 1;
  if (kind == 0) {
    if (!pi_active) return;
    const int c = t;
    if (final) {
      double s = 0.0;
      for (int p = threadIdx.x; p < m; p += blockDim.x) s += (double)X[(size_t)p * ncol + c] * Y[(size_t)p * ncol + c];
      s = block_sum(s, red);
      if (threadIdx.x == 0) sig2[t] = s;
      return;
    }
    double s = 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const double y = Y[(size_t)p * ncol + c];
      s += y * y;
    }
    s = block_sum(s, red);
    const double inv = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    for (int p = threadIdx.x; p < n2; p += blockDim.x)
      X[(size_t)p * ncol + c] = (p < m) ? (float)(Y[(size_t)p * ncol + c] * inv) : 0.f;
    return;
  }
  const int c0 = nb + 2 * t;
  if (final) {
    // S = X^T (G X) (X orthonormal), SVQB -> W = X V D^-1/2, GW = Y V D^-1/2,
    // M = (GW)^T (GW); Ritz values = eig(M)
    double s00 = 0, s01 = 0, s11 = 0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const double x0 = X[(size_t)p * ncol + c0], x1 = X[(size_t)p * ncol + c0 + 1];
      const double y0 = Y[(size_t)p * ncol + c0], y1 = Y[(size_t)p * ncol + c0 + 1];
      s00 += x0 * y0; s01 += 0.5 * (x0 * y1 + x1 * y0); s11 += x1 * y1;
    }
    s00 = block_sum(s00, red); s01 = block_sum(s01, red); s11 = block_sum(s11, red);
    // eig of the 2x2 S
    double l0, l1, v00, v01, v10, v11;
    {
      const double tr = 0.5 * (s00 + s11), df = 0.5 * (s00 - s11);
      const double rad = sqrt(df * df + s01 * s01);
      l0 = tr + rad; l1 = tr - rad;
      if (rad == 0.0) { v00 = 1; v10 = 0; v01 = 0; v11 = 1; }
      else {
        const double th = 0.5 * atan2(2.0 * s01, s00 - s11);
        v00 = cos(th); v10 = sin(th); v01 = -v10; v11 = v00;
      }
    }
    const double tol = 1e-6 * fmax(l0, 0.0);
    const double a0 = (l0 > tol && l0 > 0) ? 1.0 / sqrt(l0) : 0.0;
    const double a1 = (l1 > tol && l1 > 0) ? 1.0 / sqrt(l1) : 0.0;
    // GW columns: g_c = Y v_c a_c ; M = G W^T G W
    double m00 = 0, m01 = 0, m11 = 0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const double y0 = Y[(size_t)p * ncol + c0], y1 = Y[(size_t)p * ncol + c0 + 1];
      const double g0 = (y0 * v00 + y1 * v10) * a0, g1 = (y0 * v01 + y1 * v11) * a1;
      m00 += g0 * g0; m01 += g0 * g1; m11 += g1 * g1;
    }
    m00 = block_sum(m00, red); m01 = block_sum(m01, red); m11 = block_sum(m11, red);
    if (threadIdx.x == 0) {
      const double tr = 0.5 * (m00 + m11), df = 0.5 * (m00 - m11);
      const double rad = sqrt(df * df + m01 * m01);
      ritz[2 * t] = tr + rad;
      ritz[2 * t + 1] = (a0 > 0 && a1 > 0) ? tr - rad : 0.0;
      if (!(a0 > 0)) { ritz[2 * t] = 0.0; ritz[2 * t + 1] = 0.0; }
    }
    return;
  }
  // Euclidean SVQB of the pair, twice (second pass on the result)
  double y0s[1];
  (void)y0s;
  for (int pass = 0; pass < 2; ++pass) {
    const float* src = (pass == 0) ? Y : X;
    double s00 = 0, s01 = 0, s11 = 0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      const double a = src[(size_t)p * ncol + c0], b = src[(size_t)p * ncol + c0 + 1];
      s00 += a * a; s01 += a * b; s11 += b * b;
    }
    s00 = block_sum(s00, red); s01 = block_sum(s01, red); s11 = block_sum(s11, red);
    const double tr = 0.5 * (s00 + s11), df = 0.5 * (s00 - s11);
    const double rad = sqrt(df * df + s01 * s01);
    const double l0 = tr + rad, l1 = tr - rad;
    double v00, v01, v10, v11;
    if (rad == 0.0) { v00 = 1; v10 = 0; v01 = 0; v11 = 1; }
    else {
      const double th = 0.5 * atan2(2.0 * s01, s00 - s11);
      v00 = cos(th); v10 = sin(th); v01 = -v10; v11 = v00;
    }
    const double tol = 1e-13 * fmax(l0, 0.0);
    const double a0 = (l0 > tol && l0 > 0) ? 1.0 / sqrt(l0) : 0.0;
    const double a1 = (l1 > tol && l1 > 0) ? 1.0 / sqrt(l1) : 0.0;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      float o0 = 0.f, o1 = 0.f;
      if (p < m) {
        const double a = src[(size_t)p * ncol + c0], b = src[(size_t)p * ncol + c0 + 1];
        o0 = (float)((a * v00 + b * v10) * a0);
        o1 = (float)((a * v01 + b * v11) * a1);
      }
      X[(size_t)p * ncol + c0] = o0;
      X[(size_t)p * ncol + c0 + 1] = o1;
    }
    __syncthreads();
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

// ---- FP64 single-row path pieces (any buffer size) --------------------------
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

// x <- y / ||y|| (first m entries); flag[0] = 1 if ||y|| == 0.  One block.
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

// One block: S = X^T X (or X^T Xg for the G inner product when gram_of != nullptr),
// SVQB with eig(S); X, Xg <- (.) V D^-1/2 (kept columns).  Rows >= m are zero.
__global__ void svqb_kernel(int n2, int m, int k, double* X, double* Xg, int g_inner, double* S, double* V,
                            double* D, double* eigw, double* tmp) {
  __shared__ double red[32];
  const double* B = g_inner ? Xg : X;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double acc = 0.0;
    for (int p = 0; p < m; ++p) acc += X[(size_t)p * k + a] * B[(size_t)p * k + c];
    S[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    if (a < c) { const double v = 0.5 * (S[a * k + c] + S[c * k + a]); S[a * k + c] = v; S[c * k + a] = v; }
  }
  __syncthreads();
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

// One block: with W (n2 x k) G-orthonormal and GW: M = GW^T GW, eig -> ritz (descending),
// WU = W U, GWU = GW U.
__global__ void rayleigh_ritz_kernel(int n2, int m, int k, const double* W, const double* GW, double* M,
                                     double* U, double* ritz, double* eigw, double* WU, double* GWU, int* status) {
  __shared__ double red[32];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double acc = 0.0;
    for (int p = 0; p < m; ++p) acc += GW[(size_t)p * k + a] * GW[(size_t)p * k + c];
    M[e] = acc;
  }
  __syncthreads();
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

__global__ void promote_pair_kernel(const float* X, int ldx, int col0, int n2, int m, int k, double* Y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 * k; e += gridDim.x * blockDim.x) {
    const int p = e / k, c = e - p * k;
    Y[e] = (p < m) ? (double)X[(size_t)p * ldx + col0 + c] : 0.0;
  }
}

}  // namespace

as_status launch_si_rr_from_batch(cudaStream_t s, const double* G, int n2, int m, const float* X, int ldx, int col0,
                                  const SiBuffers& b, int* status) {
  const int k = 2;
  promote_pair_kernel<<<(n2 * k + 255) / 256, 256, 0, s>>>(X, ldx, col0, n2, m, k, b.Y); count_launches(1);
  AS_CUDA_TRY(cudaMemsetAsync(b.GY, 0, (size_t)n2 * k * sizeof(double), s));
  as_status st = gemm_strided<double, double, double>(s, m, k, m, G, n2, 1, b.Y, k, 1, b.GY, k, 1, 1.0, 0.0);
  if (st != AS_OK) return st;
  svqb_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, 1, b.S, b.V, b.ritz, b.eigw, b.tmp); count_launches(1);
  rayleigh_ritz_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, b.S, b.V, b.ritz, b.eigw, b.WU, b.GWU, status); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_gf_mirror(cudaStream_t s, const double* G, float* Gf, int n2, int m) {
  const size_t tot = (size_t)n2 * n2;
  const int blocks = (int)std::min<size_t>((tot + 255) / 256, 4096);
  mirror_f32_kernel<<<blocks, 256, 0, s>>>(G, Gf, n2, m); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_batch_gspace(cudaStream_t s, const float* Gf, int n2, int r0, int nb, int k_pi, int q, Key key,
                              uint64_t i0, const BatchBuffers& bb, Prof* prof) {
  if (nb <= 0) return AS_OK;
  const int ncol = 3 * nb;
  const int mmax = r0 + nb;
  batch_fill_kernel<<<dim3(nb, 2), 128, 0, s>>>(bb.X, n2, ncol, nb, r0, key, i0); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  const int iters = std::max(k_pi, q);
  for (int it = 0; it <= iters; ++it) {
    const bool pi_on = it <= k_pi;
    const bool si_on = it <= q;
    const int c0 = pi_on ? 0 : nb;
    const int c1 = si_on ? ncol : nb;
    if (prof) prof->begin(PK_BATCH_GEMM, s);
    as_status st = gemm_strided<float, float, float>(s, mmax, c1 - c0, mmax, Gf, n2, 1, bb.X + c0, ncol, 1,
                                                     bb.Y + c0, ncol, 1, 1.0, 0.0);
    if (st != AS_OK) return st;
    // algorithmic work of one product: 2 m^2 N flops; G (m^2 FP32) read once, X read, Y written
    if (prof)
      prof->end(PK_BATCH_GEMM, s, 2.0 * mmax * (double)mmax * (c1 - c0),
                4.0 * ((double)mmax * mmax + 2.0 * (double)mmax * (c1 - c0)));
    if (prof) prof->begin(PK_BATCH_ORTH, s);
    // PI: iterations 0..k_pi-1 normalise, iteration k_pi evaluates sigma^2.
    // SI: iterations 0..q-1 orthonormalise, iteration q does Rayleigh-Ritz.
    if (pi_on) {
      batch_orth_kernel<<<dim3(nb, 1), 256, 0, s>>>(bb.Y, bb.X, n2, ncol, nb, r0, 1, it == k_pi ? 1 : 0,
                                                    bb.sig2, bb.ritz); count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
    }
    if (si_on) {
      // the SI pair's kernel instance is selected by blockIdx.y = 1
      batch_orth_kernel<<<dim3(nb, 2), 256, 0, s>>>(bb.Y, bb.X, n2, ncol, nb, r0, 0, it == q ? 1 : 0, bb.sig2,
                                                    bb.ritz); count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
    }
    if (prof) prof->end(PK_BATCH_ORTH, s, 0.0, 8.0 * (double)mmax * (c1 - c0));
  }
  return AS_OK;
}

as_status launch_power_iteration_f64(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key,
                                     uint64_t i, double* x, double* y, int* zero, double* sig2) {
  AS_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(int), s));
  fill_pi_start<<<(n2 / 4 + 255) / 256 + 1, 256, 0, s>>>(x, n2, m, key, i); count_launches(1);
  normalize_kernel<<<1, 512, 0, s>>>(x, x, m, zero); count_launches(1);
  for (int it = 0; it < k_pi; ++it) {
    as_status st = gemm_strided<double, double, double>(s, m, 1, m, G, n2, 1, x, 1, 1, y, 1, 1, 1.0, 0.0);
    if (st != AS_OK) return st;
    normalize_kernel<<<1, 512, 0, s>>>(y, x, m, zero); count_launches(1);
  }
  as_status st = gemm_strided<double, double, double>(s, m, 1, m, G, n2, 1, x, 1, 1, y, 1, 1, 1.0, 0.0);
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
    as_status st = gemm_strided<double, double, double>(s, m, k, m, G, n2, 1, b.Y, k, 1, b.GY, k, 1, 1.0, 0.0);
    if (st != AS_OK) return st;
    for (int pass = 0; pass < 2; ++pass) {
      svqb_kernel<<<1, 512, 0, s>>>(n2, m, k, b.GY, nullptr, 0, b.S, b.V, b.ritz, b.eigw, b.tmp); count_launches(1);
    }
    AS_CUDA_TRY(cudaMemcpyAsync(b.Y, b.GY, (size_t)n2 * k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  as_status st = gemm_strided<double, double, double>(s, m, k, m, G, n2, 1, b.Y, k, 1, b.GY, k, 1, 1.0, 0.0);
  if (st != AS_OK) return st;
  svqb_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, 1, b.S, b.V, b.ritz, b.eigw, b.tmp); count_launches(1);
  rayleigh_ritz_kernel<<<1, 512, 0, s>>>(n2, m, k, b.Y, b.GY, b.S, b.V, b.ritz, b.eigw, b.WU, b.GWU, status); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
