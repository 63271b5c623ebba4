// The FP64 single-row path of the G-space iterations for large buffers
// (power iteration, simultaneous iteration, Rayleigh-Ritz from the batched
// basis), the incremental FP32 mirror of G read by the batched iterations
// (batch_persist.cu), and the dump kernels (the snapshot and residual step of Algorithm 4).
#include <algorithm>

#include "eig.cuh"
#include "grid.cuh"
#include "kernels.cuh"

namespace as {

namespace {

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

// Gf (FP32) = G (FP64) on the rows/columns of the leading m x m block that
// are not yet mirrored: row p (one CTA per row) gets columns [valid, m) when
// p < valid and [0, m) otherwise.
__global__ void mirror_strip_kernel(const double* G, float* Gf, int n2, int valid, int m) {
  const int p = blockIdx.x;
  if (p >= m) return;
  const int q0 = (p < valid) ? valid : 0;
  const double* g = G + (size_t)p * n2;
  float* f = Gf + (size_t)p * n2;
  for (int q = q0 + threadIdx.x; q < m; q += blockDim.x) f[q] = (float)g[q];
}

// ---- FP64 single-row path (any buffer size) ---------------------------------
__global__ void fill_pi_start(double* x, int n2, int m, Key key, uint64_t i, uint64_t jsub) {
  for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < n2; blk += gridDim.x * blockDim.x) {
    double z[4];
    gauss4(key, kPurposePiStart, i, jsub, blk, z);
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

// S = sym(A^T B) over the first m rows (A, B row-major n2 x k), for k = K
// known at compile time: every thread accumulates the K (K + 1) / 2 entries
// over its rows in one pass (a row's K values are contiguous), and the
// entries are then reduced together, each in the order of block_sum: a warp
// butterfly, then warp 0 over the warps' sums.  FP64 issue is scarce on this
// part, so no entry beyond k is computed.
template <int K>
__device__ void block_gram_k(int m, const double* A, const double* B, double* S) {
  constexpr int kT = K * (K + 1) / 2;
  __shared__ double wsum[32][kT];
  double acc[kT];
#pragma unroll
  for (int t = 0; t < kT; ++t) acc[t] = 0.0;
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    double ar[K], br[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
      ar[a] = A[(size_t)p * K + a];
      br[a] = B[(size_t)p * K + a];
    }
    int t = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int c = a; c < K; ++c, ++t) acc[t] += 0.5 * (ar[a] * br[c] + ar[c] * br[a]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int t = 0; t < kT; ++t) {
    const double v = warp_sum(acc[t]);
    if (lane == 0) wsum[wid][t] = v;
  }
  __syncthreads();
  if (wid == 0) {
    int t = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int c = a; c < K; ++c, ++t) {
        const double v = warp_sum((lane < nw) ? wsum[lane][t] : 0.0);
        if (lane == 0) { S[a * K + c] = v; S[c * K + a] = v; }
      }
  }
  __syncthreads();
}

__device__ void block_gram(int m, int k, const double* A, const double* B, double* S, double* red) {
  if (k == 2) { block_gram_k<2>(m, A, B, S); return; }
  if (k == 4) { block_gram_k<4>(m, A, B, S); return; }
  if (k == 8) { block_gram_k<8>(m, A, B, S); return; }
  if (k < 8) {
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
__global__ void __launch_bounds__(512) svqb_kernel(int n2, int m, int k, double* X, double* Xg, int g_inner, double* S, double* V,
                            double* D, double* eigw, double* tmp) {
  __shared__ double red[32];
  block_gram(m, k, X, g_inner ? Xg : X, S, red);
  EigWork w = eig_work_view(eigw, k, k);
  cta_eig_sym(k, S, k, k, D, V, k, w, red);
  __syncthreads();
  const double dmax = D[0];
  // 1 / sqrt(D_c) once per column (0 for a numerically null direction)
  __shared__ double rs[64];
  for (int c = threadIdx.x; c < k && c < 64; c += blockDim.x)
    rs[c] = (dmax > 0.0 && D[c] > 1e-13 * dmax) ? 1.0 / sqrt(D[c]) : 0.0;
  __syncthreads();
  const int passes = Xg ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    double* M = (pass == 0) ? X : Xg;
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      for (int c = 0; c < k; ++c) {
        double acc = 0.0;
        const double sc = (c < 64) ? rs[c] : ((dmax > 0.0 && D[c] > 1e-13 * dmax) ? 1.0 / sqrt(D[c]) : 0.0);
        if (p < m && sc != 0.0) {
          for (int a = 0; a < k; ++a) acc += M[(size_t)p * k + a] * V[a * k + c];
          acc *= sc;
        }
        tmp[(size_t)p * k + c] = acc;
      }
      for (int c = 0; c < k; ++c) M[(size_t)p * k + c] = tmp[(size_t)p * k + c];
    }
    __syncthreads();
  }
}

// One block: with W G-orthonormal and GW: M = GW^T GW, eig -> ritz (descending), WU, GWU.
__global__ void __launch_bounds__(512) rayleigh_ritz_kernel(int n2, int m, int k, const double* W, const double* GW, double* M, double* U,
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

// Rayleigh-Ritz of Algorithm 2 for k = 2 in FP64, closed-form 2 x 2
// eigenproblems: S = Y^T (G Y) = V D V^T, W = Y V D^-1/2, GW = (G Y) V D^-1/2,
// M = GW^T GW = U diag(ritz) U^T, WU, GWU.  Y is orthonormal (Euclidean).
// The pair sums are FP64 multiply-adds, and one SM's FP64 issue rate would
// make a single block take tens of microseconds at m = 2048, so the rows are
// spread over several blocks (one cooperative launch): each block forms
// partial sums over its share, and after a grid barrier every block adds the
// partials in block order, so that every block holds the same coefficients.
__global__ void __launch_bounds__(256) rr2_coop_kernel(int n2, int m, const double* Y, const double* GY,
                                                        double* ritz, double* WU, double* GWU, double* part,
                                                        unsigned* cnt, int* status) {
  __shared__ double red[32];
  __shared__ double cf[8];
  const int G = gridDim.x, tid = threadIdx.x, stride = G * blockDim.x;
  double s00 = 0, s01 = 0, s11 = 0;
  for (int p = blockIdx.x * blockDim.x + tid; p < m; p += stride) {
    const double a = Y[2 * p], b = Y[2 * p + 1], ga = GY[2 * p], gb = GY[2 * p + 1];
    s00 += a * ga; s01 += 0.5 * (a * gb + b * ga); s11 += b * gb;
  }
  s00 = block_sum(s00, red); s01 = block_sum(s01, red); s11 = block_sum(s11, red);
  if (tid == 0) { part[3 * blockIdx.x] = s00; part[3 * blockIdx.x + 1] = s01; part[3 * blockIdx.x + 2] = s11; }
  if (!grid_barrier(cnt, (unsigned)G, status)) return;
  if (tid == 0) {
    double t00 = 0, t01 = 0, t11 = 0;
    for (int g = 0; g < G; ++g) { t00 += part[3 * g]; t01 += part[3 * g + 1]; t11 += part[3 * g + 2]; }
    double l0, l1, v00, v01, v10, v11;
    eig2(t00, t01, t11, l0, l1, v00, v01, v10, v11);
    const double a0 = (l0 > 0.0) ? 1.0 / sqrt(l0) : 0.0;
    const double a1 = (l1 > 1e-13 * l0 && l1 > 0.0) ? 1.0 / sqrt(l1) : 0.0;
    cf[0] = v00 * a0; cf[1] = v10 * a0; cf[2] = v01 * a1; cf[3] = v11 * a1;
  }
  __syncthreads();
  const double w00 = cf[0], w10 = cf[1], w01 = cf[2], w11 = cf[3];
  double m00 = 0, m01 = 0, m11 = 0;
  for (int p = blockIdx.x * blockDim.x + tid; p < m; p += stride) {
    const double ga = GY[2 * p], gb = GY[2 * p + 1];
    const double g0 = ga * w00 + gb * w10, g1 = ga * w01 + gb * w11;
    m00 += g0 * g0; m01 += g0 * g1; m11 += g1 * g1;
  }
  m00 = block_sum(m00, red); m01 = block_sum(m01, red); m11 = block_sum(m11, red);
  double* part2 = part + 3 * G;
  if (tid == 0) { part2[3 * blockIdx.x] = m00; part2[3 * blockIdx.x + 1] = m01; part2[3 * blockIdx.x + 2] = m11; }
  if (!grid_barrier(cnt, 2u * (unsigned)G, status)) return;
  if (tid == 0) {
    double t00 = 0, t01 = 0, t11 = 0;
    for (int g = 0; g < G; ++g) { t00 += part2[3 * g]; t01 += part2[3 * g + 1]; t11 += part2[3 * g + 2]; }
    double r0, r1, u00, u01, u10, u11;
    eig2(t00, t01, t11, r0, r1, u00, u01, u10, u11);
    if (blockIdx.x == 0) {
      ritz[0] = r0;
      ritz[1] = (w01 != 0.0 || w11 != 0.0) ? r1 : 0.0;
      if (!(r0 == r0)) set_status(status, AS_ENUMERIC);
    }
    cf[4] = u00; cf[5] = u10; cf[6] = u01; cf[7] = u11;
  }
  __syncthreads();
  const double u00 = cf[4], u10 = cf[5], u01 = cf[6], u11 = cf[7];
  for (int p = blockIdx.x * blockDim.x + tid; p < n2; p += stride) {
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

// ---- dump (snapshot and residual, Algorithm 4) -------------------------------
// Partial sums over row chunks s: Zp[s][c][a - ab] = sum_p C[p][c] WU[p][a] and
// Yp[s][a - ab][c] = sum_p GWU[p][a] C[p][c] for a in [a0, a0+na) inside the
// column block [ab, ab + w), one thread per column c.  Blocks of at most
// kDumpBlock snapshot columns bound the partial planes whatever xi is.  Narrow
// blocks (the usual snapshot ranks) take more row chunks, so that enough loads
// of C are in flight to stream it at memory speed.
constexpr int kDumpBlock = 64;
__host__ __device__ constexpr int dump_chunks(int w) { return w <= 16 ? 32 : 8; }
// columns of one partial plane set: the largest w * dump_chunks(w) over the
// column blocks of a rank-xi snapshot
inline size_t dump_plane_cols(int xi) {
  const int w1 = std::min(xi, kDumpBlock);
  return (size_t)std::max(std::min(xi, 16) * dump_chunks(std::min(xi, 16)), w1 * dump_chunks(w1));
}

// FP32 copies of the first xi columns of WU and GWU (rows < r, row-major
// r x xi), and the low part GWUlo = fl32(GWU - GWUf) for the residual.
// Converting once keeps FP64 work out of the per-entry loops below.
__global__ void dump_coef_f32(const double* WU, const double* GWU, int r, int k, int xi, float* WUf, float* GWUf,
                              float* GWUlo) {
  const int tot = r * xi;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int p = e / xi, a = e - p * xi;
    const double g = GWU[(size_t)p * k + a];
    const float gf = (float)g;
    WUf[e] = (float)WU[(size_t)p * k + a];
    GWUf[e] = gf;
    GWUlo[e] = (float)(g - (double)gf);
  }
}

__global__ void dump_partial_kernel(const float* __restrict__ C, int ldc, int d, int r, const float* __restrict__ WUf,
                                    const float* __restrict__ GWUf, int xi, int a0, int na, int ab, int w, double* Zp,
                                    double* Yp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, nch = gridDim.y;
  if (c >= d) return;
  const int chunk = (r + nch - 1) / nch;
  const int pb = s * chunk, pe = min(r, pb + chunk);
  double z[8], y[8];
  float zf[8], yf[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) { z[a] = 0.0; y[a] = 0.0; zf[a] = 0.f; yf[a] = 0.f; }
  int cnt = 0;
  // eight rows at a time: their loads of C go out together (one load per row
  // and thread would leave the kernel waiting on memory latency)
  for (int p8 = pb; p8 < pe; p8 += 8) {
    float cv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) cv[u] = (p8 + u < pe) ? C[(size_t)(p8 + u) * ldc + c] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = p8 + u;
      if (p < pe) {
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < na) {
            zf[a] = fmaf(cv[u], WUf[(size_t)p * xi + a0 + a], zf[a]);
            yf[a] = fmaf(cv[u], GWUf[(size_t)p * xi + a0 + a], yf[a]);
          }
        if (++cnt == 64) {   // FP32 partial sums of 64 rows, combined in FP64
          cnt = 0;
#pragma unroll
          for (int a = 0; a < 8; ++a) { z[a] += zf[a]; y[a] += yf[a]; zf[a] = 0.f; yf[a] = 0.f; }
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a)
    if (a < na) {
      Zp[((size_t)s * d + c) * w + (a0 - ab) + a] = z[a] + zf[a];
      Yp[((size_t)s * w + (a0 - ab) + a) * d + c] = y[a] + yf[a];
    }
}

// Columns [ab, ab + w) of Z (d x xi row-major) and rows [ab, ab + w) of Y
// (xi x d row-major) from the block's partial planes.
__global__ void dump_reduce_kernel(const double* Zp, const double* Yp, int d, int xi, int ab, int w, float* Z,
                                   float* Y) {
  const int tot = d * w, nch = dump_chunks(w);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    double z = 0.0, y = 0.0;
    for (int s = 0; s < nch; ++s) { z += Zp[(size_t)s * tot + e]; y += Yp[(size_t)s * tot + e]; }
    const int c = e / w, a = e - c * w;
    Z[(size_t)c * xi + ab + a] = (float)z;   // Zp element e = c*w + a
    Y[(size_t)ab * d + e] = (float)y;        // Yp element e = a*d + c
  }
}

// C[p][c] -= sum_a GWU[p][a] Z[c][a]   (the residual C' - C' Z Z^T), as an
// FMA chain in FP32 with GWU split into hi + lo: each term enters with one
// rounding, so a strongly cancelling entry keeps its relative accuracy.
// With the tensor forms, the BF16 levels of the new entries (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); l2 may be null) are written in
// the same pass.
__global__ void residual_kernel(float* C, int ldc, int d, int r, const float* __restrict__ GWUf,
                                const float* __restrict__ GWUlo, int xi, const float* Z, __nv_bfloat16* l0,
                                __nv_bfloat16* l1, __nv_bfloat16* l2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (c >= d || p >= r) return;
  float v = C[(size_t)p * ldc + c];
  for (int a = 0; a < xi; ++a) {
    const float z = Z[(size_t)c * xi + a];
    v = fmaf(-GWUf[(size_t)p * xi + a], z, v);
    v = fmaf(-GWUlo[(size_t)p * xi + a], z, v);
  }
  const size_t o = (size_t)p * ldc + c;
  C[o] = v;
  if (l0) {
    const __nv_bfloat16 a0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(a0);
    const __nv_bfloat16 a1 = __float2bfloat16_rn(r1);
    l0[o] = a0;
    l1[o] = a1;
    if (l2) l2[o] = __float2bfloat16_rn(r1 - __bfloat162float(a1));
  }
}

// R[p][q] = G[p][q] - sum_{a < xi} GWU[p][a] GWU[q][a] for p, q < m (the Gram
// of the residual C' - C' Z Z^T, Z the first xi columns), into R (ld n2).
__global__ void residual_gram_kernel(const double* G, int n2, int m, const double* GWU, int k, int xi, double* R) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (q >= m || p >= m) return;
  double acc = G[(size_t)p * n2 + q];
  for (int a = 0; a < xi; ++a) acc -= GWU[(size_t)p * k + a] * GWU[(size_t)q * k + a];
  R[(size_t)p * n2 + q] = acc;
}

// G[p][q] -= sum_a GWU[p][a] GWU[q][a], and the same entries of the FP32
// mirror (Gf, ld n2) and of the BF16 levels (Gb, ld ldg, glevel apart) when given.
__global__ void gram_downdate_kernel(double* G, int n2, int r, const double* GWU, int k, int xi, float* Gf,
                                     __nv_bfloat16* Gb, long long glevel, int ldg) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (q >= r || p >= r) return;
  double acc = 0.0;
  for (int a = 0; a < xi; ++a) acc += GWU[(size_t)p * k + a] * GWU[(size_t)q * k + a];
  const double x = G[(size_t)p * n2 + q] - acc;
  G[(size_t)p * n2 + q] = x;
  if (Gf) Gf[(size_t)p * n2 + q] = (float)x;
  if (Gb) {
    __nv_bfloat16 b0, b1, b2;
    g_levels(x, b0, b1, b2);
    __nv_bfloat16* o = Gb + (size_t)p * ldg + q;
    o[0] = b0;
    o[glevel] = b1;
    o[2 * glevel] = b2;
  }
}

}  // namespace

as_status launch_gf_mirror(cudaStream_t s, const double* G, float* Gf, int n2, int valid, int m) {
  if (m <= 0 || valid >= m) return AS_OK;
  mirror_strip_kernel<<<m, 256, 0, s>>>(G, Gf, n2, std::max(valid, 0), m); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

static as_status gmul_thin(cudaStream_t s, const double* G, int n2, int m, int k, const double* X, double* Y) {
  if (m <= 0) return AS_OK;   // an empty buffer: no rows of Y to form
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
  if (m <= 0) return AS_OK;
  if (k <= 8) return gmul_thin(s, G, n2, m, k, X, Y);
  return gemm_strided<double, double, double>(s, m, k, m, G, n2, 1, X, k, 1, Y, k, 1, 1.0, 0.0);
}

as_status launch_power_iteration_f64(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key, uint64_t i,
                                     double* x, double* y, int* zero, double* sig2, uint64_t jsub) {
  if (m <= 0) {   // an empty buffer (after the shrink of l = 1): sigma_hat^2 = 0
    AS_CUDA_TRY(cudaMemsetAsync(sig2, 0, sizeof(double), s));
    return AS_OK;
  }
  AS_CUDA_TRY(cudaMemsetAsync(zero, 0, sizeof(int), s));
  fill_pi_start<<<(n2 / 4 + 255) / 256 + 1, 256, 0, s>>>(x, n2, m, key, i, jsub); count_launches(1);
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
  // up to 16 blocks of 256 rows each; the partial sums (6 per block) and the
  // barrier counter live in the free scratch b.tmp (n2 * 2 + 14 doubles or
  // more, enough for 6 * ceil(n2 / 256) + 1)
  const int nblk = std::max(1, std::min(16, (m + 255) / 256));
  double* part = b.tmp;
  unsigned* cnt = reinterpret_cast<unsigned*>(b.tmp + 6 * nblk);
  AS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
  int n2a = n2, ma = m;
  const double* Ya = b.Y;
  const double* GYa = b.GY;
  double *ra = b.ritz, *wua = b.WU, *gwua = b.GWU;
  int* sta = status;
  void* args[] = {&n2a, &ma, &Ya, &GYa, &ra, &wua, &gwua, &part, &cnt, &sta};
  AS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)rr2_coop_kernel, dim3(nblk), dim3(256), args, 0, s));
  count_launches(1);
  return AS_OK;
}

as_status launch_residual_gram(cudaStream_t s, const double* G, int n2, int m, const double* GWU, int k, int xi,
                               double* R) {
  if (m <= 0) return AS_OK;
  residual_gram_kernel<<<dim3((m + 255) / 256, m), 256, 0, s>>>(G, n2, m, GWU, k, xi, R); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

size_t dump_work_doubles(int d, int n2, int xi) {
  // partial planes of one column block + the FP32 coefficients
  return (size_t)2 * d * dump_plane_cols(xi) + ((size_t)3 * n2 * xi + 1) / 2;
}

as_status launch_dump(cudaStream_t s, float* C, int ldc, int d, int r, double* G, int n2, const double* WU,
                      const double* GWU, int k, int xi, float* Z, float* Y, double* work, const DumpMirrors& mir) {
  const size_t plane = (size_t)d * dump_plane_cols(xi);   // doubles of each of Zp, Yp
  double* Zp = work;
  double* Yp = work + plane;
  float* WUf = reinterpret_cast<float*>(Yp + plane);
  float* GWUf = WUf + (size_t)n2 * xi;
  float* GWUlo = GWUf + (size_t)n2 * xi;
  if (r > 0) {
    dump_coef_f32<<<(r * xi + 255) / 256, 256, 0, s>>>(WU, GWU, r, k, xi, WUf, GWUf, GWUlo); count_launches(1);
  }
  for (int ab = 0; ab < xi; ab += kDumpBlock) {
    const int w = std::min(kDumpBlock, xi - ab);
    for (int a0 = ab; a0 < ab + w; a0 += 8) {
      const int na = std::min(8, ab + w - a0);
      dim3 grid((d + 127) / 128, dump_chunks(w));
      dump_partial_kernel<<<grid, 128, 0, s>>>(C, ldc, d, r, WUf, GWUf, xi, a0, na, ab, w, Zp, Yp);
      count_launches(1);
    }
    dump_reduce_kernel<<<(d * w + 255) / 256, 256, 0, s>>>(Zp, Yp, d, xi, ab, w, Z, Y); count_launches(1);
  }
  if (r > 0) {
    residual_kernel<<<dim3((d + 255) / 256, r), 256, 0, s>>>(C, ldc, d, r, GWUf, GWUlo, xi, Z, mir.c0, mir.c1,
                                                             mir.c2);
    count_launches(1);
    gram_downdate_kernel<<<dim3((r + 255) / 256, r), 256, 0, s>>>(G, n2, r, GWU, k, xi, mir.gf, mir.gb, mir.glevel,
                                                                  mir.ldg);
    count_launches(1);
  }
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
