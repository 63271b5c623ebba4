// The low-rank route of the query (Algorithm 5).
//
// The query matrix is B = C^T C + sum_j (Z_j Y_j + Y_j^T Z_j^T - Z_j (Y_j Z_j) Z_j^T).
// Stacking the factors as the rows of F = [C; Z_1^T; Y_1; Z_2^T; Y_2; ...]
// (r_F x d) gives B = F^T H F with a small block-diagonal H: the identity on
// the rows of C and, for snapshot j,
//     H_j = [[-Y_j Z_j, I], [I, 0]],
// because [Z  Y^T] H_j [Z^T; Y] = Z Y + Y^T Z^T - Z (Y Z) Z^T.  When r_F < d the
// eigenpairs of B come from r_F x r_F problems instead of the d x d one:
//   1. W = F F^T, scaled to unit diagonal: W' = D W D, D = diag(W_ii^-1/2);
//      H' = D^-1 H D^-1, so that B = F^T D H' D F.  Y_j Z_j is the block of W
//      between the rows of Y_j and those of Z_j^T, so H' comes from W.
//   2. W' = U L U^T; the r' eigenvalues above a relative cutoff span the row
//      space of D F (the rest is numerically null), and
//      Q = F^T D U_r L_r^-1/2 has orthonormal columns spanning it.
//   3. K = Q^T B Q = L_r^1/2 U_r^T H' U_r L_r^1/2 (r' x r', because
//      W' U_r = U_r L_r), K = U_k M U_k^T.
//   4. The eigenpairs of B outside null(F) are (M, Q U_k), with
//      Q U_k = F^T E, E = D U_r L_r^-1/2 U_k.  B is zero on null(F), which has
//      dimension d - r' > 0, so the l-th largest eigenvalue of B is
//      max(M_l, 0) (0 when r' < l).
// The eigensolvers are those of the dense route; FP64 throughout except F,
// which holds the stored FP32 values.
#include "kernels.cuh"

namespace as {

namespace {

// out (xi x d, row-major, ld ldo) = Z^T for Z (d x xi, row-major).
__global__ void transpose_f32_kernel(const float* Z, int d, int xi, float* out, long long ldo) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;   // c over d, r over xi
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (c < d && r < xi) ? Z[(size_t)c * xi + r] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    if (r < xi && c < d) out[(size_t)r * ldo + c] = tile[threadIdx.x][y];
  }
}

// W' = D W D and H' = D^-1 H D^-1 (both n x n, row-major) from W = F F^T.
// kind[i] = {type, oz, xi}: type 0 a row of C, 1 row a of Z_j^T, 2 row a of
// Y_j, with oz the first row of Z_j^T and xi the snapshot's rank (the rows of
// Y_j start at oz + xi).
__global__ void lr_scale_kernel(const double* W, int n, const int4* kind, double* Ws, double* Hs) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const double wii = W[(size_t)i * n + i];
  const double di = (wii > 0.0) ? rsqrt(wii) : 0.0, si = (wii > 0.0) ? sqrt(wii) : 0.0;
  const int4 ki = kind[i];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double wjj = W[(size_t)j * n + j];
    const double dj = (wjj > 0.0) ? rsqrt(wjj) : 0.0, sj = (wjj > 0.0) ? sqrt(wjj) : 0.0;
    Ws[(size_t)i * n + j] = W[(size_t)i * n + j] * di * dj;
    double h = 0.0;
    if (ki.x == 0) {
      h = (j == i) ? 1.0 : 0.0;
    } else if (j >= ki.y && j < ki.y + 2 * ki.z) {
      const int a = (ki.x == 1) ? i - ki.y : i - ki.y - ki.z;   // index inside the snapshot
      const int b = j - ki.y;                                  // < xi: a Z row; else a Y row
      if (ki.x == 1 && b < ki.z) {
        // -(Y Z)[a][b] = -W[row of Y_a][row of Z^T_b]
        h = -W[(size_t)(ki.y + ki.z + a) * n + (ki.y + b)];
      } else if (ki.x == 1) {
        h = (b - ki.z == a) ? 1.0 : 0.0;
      } else {
        h = (b == a) ? 1.0 : 0.0;
      }
    }
    Hs[(size_t)i * n + j] = h * si * sj;
  }
}

// K[i][j] = 0.5 (T[i][j] + T[j][i]) sqrt(lam_i lam_j) for i, j < r (ld ldk).
__global__ void lr_core_kernel(const double* T, int ldt, const double* lam, int r, double* K) {
  const int i = blockIdx.x;
  if (i >= r) return;
  const double li = sqrt(fmax(lam[i], 0.0));
  for (int j = threadIdx.x; j < r; j += blockDim.x)
    K[(size_t)i * r + j] = 0.5 * (T[(size_t)i * ldt + j] + T[(size_t)j * ldt + i]) * li * sqrt(fmax(lam[j], 0.0));
}

// E[i][c] = d_i * P[i][c] with P = U_r L_r^-1/2 U_k already formed as
// (U_r diag(lam^-1/2)) U_k: here the row scaling by D of the n x m matrix P.
__global__ void lr_rowscale_kernel(const double* W, int n, double* P, int m) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const double wii = W[(size_t)i * n + i];
  const double di = (wii > 0.0) ? rsqrt(wii) : 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) P[(size_t)i * m + c] *= di;
}

// U[i][c] *= lam_c^-1/2 for c < r (U is n x ldu, row-major).
__global__ void lr_colscale_kernel(double* U, int n, int ldu, const double* lam, int r) {
  const int i = blockIdx.x;
  if (i >= n) return;
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const double l = lam[c];
    U[(size_t)i * ldu + c] *= (l > 0.0) ? rsqrt(l) : 0.0;
  }
}

// lam_out[0..l) = the l largest eigenvalues of B: mu[0..l') then zeros, with
// the l-th raised to max(mu_l, 0) (B is zero on the null space of F).
__global__ void lr_lambda_kernel(const double* mu, int lp, int ell, double* lam_out) {
  for (int i = threadIdx.x; i < ell; i += blockDim.x) {
    double v = (i < lp) ? mu[i] : 0.0;
    if (i == ell - 1) v = fmax(v, 0.0);
    lam_out[i] = v;
  }
}

__global__ void f32_to_f64_kernel(const float* in, size_t n, double* out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

}  // namespace

as_status launch_f32_to_f64(cudaStream_t s, const float* in, size_t n, double* out) {
  if (n == 0) return AS_OK;
  f32_to_f64_kernel<<<1024, 256, 0, s>>>(in, n, out);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_transpose_f32(cudaStream_t s, const float* Z, int d, int xi, float* out, long long ldo) {
  if (d <= 0 || xi <= 0) return AS_OK;
  dim3 grid((d + 31) / 32, (xi + 31) / 32), block(32, 8);
  transpose_f32_kernel<<<grid, block, 0, s>>>(Z, d, xi, out, ldo);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_lr_scale(cudaStream_t s, const double* W, int n, const int4* kind, double* Ws, double* Hs) {
  if (n <= 0) return AS_OK;
  lr_scale_kernel<<<n, 256, 0, s>>>(W, n, kind, Ws, Hs);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_lr_core(cudaStream_t s, const double* T, int ldt, const double* lam, int r, double* K) {
  if (r <= 0) return AS_OK;
  lr_core_kernel<<<r, 256, 0, s>>>(T, ldt, lam, r, K);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_lr_colscale(cudaStream_t s, double* U, int n, int ldu, const double* lam, int r) {
  if (n <= 0 || r <= 0) return AS_OK;
  lr_colscale_kernel<<<n, 256, 0, s>>>(U, n, ldu, lam, r);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_lr_rowscale(cudaStream_t s, const double* W, int n, double* P, int m) {
  if (n <= 0 || m <= 0) return AS_OK;
  lr_rowscale_kernel<<<n, 256, 0, s>>>(W, n, P, m);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

as_status launch_lr_lambda(cudaStream_t s, const double* mu, int lp, int ell, double* lam_out) {
  lr_lambda_kernel<<<1, 256, 0, s>>>(mu, lp, ell, lam_out);
  count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
