// Launchers of the AeroSketch kernels (internal C++ interface of the library).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace as {

// Strided SIMT GEMM, see gemm.cu.
template <typename TA, typename TB, typename TO>
as_status gemm_strided(cudaStream_t s, int M, int N, int K, const TA* A, long long sam, long long sak,
                       const TB* B, long long sbk, long long sbn, TO* O, long long som, long long son,
                       double alpha, double beta);

// Copy n rows (ld_in) into C rows [r, r+n) (ldc, FP32) and write each row's
// squared norm (FP64) to norm2[t]; a non-finite value sets *bad = 1.
as_status launch_ingest(cudaStream_t s, const float* rows, long long ld_in, int n, int d, float* C,
                        int ldc, int r, double* norm2, int* bad);

// Zero rows [r0, r1) of C (ldc) and rows/columns [r0, n2) of G (n2 x n2).
as_status launch_truncate(cudaStream_t s, float* C, int ldc, int d, int r0, int r1, double* G, int n2);

// G[p][r+t] for p < r+b, t < b from the new rows, then mirror to G[r+t][p].
as_status launch_gram_rows(cudaStream_t s, const float* C, int ldc, int d, int r, int b, double* G, int n2);

// Algorithm 1 on C' via G = C' C'^T restricted to the first m rows; writes
// sigma_hat_1^2 to *sig2.
as_status launch_power_iteration(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key,
                                 uint64_t i, double* sig2);

struct SiBuffers {
  double* Y;      // n2 x kmax
  double* GY;     // n2 x kmax
  double* S;      // kmax x kmax
  double* V;      // kmax x kmax
  double* eigw;   // eig_work_doubles(kmax, kmax)
  double* ritz;   // kmax
  double* WU;     // n2 x kmax  (coefficients of Z = C'^T WU)
  double* GWU;    // n2 x kmax  (G WU; Y_snap = GWU^T C')
  double* tmp;    // n2 * kmax + 3 * kmax^2 + kmax
};

// Algorithm 2 on C' via G (first m rows), k columns, q products, test
// matrix from Philox (purpose 4, i, j).  Writes ritz[0..k) descending, WU, GWU.
as_status launch_simul_iter(cudaStream_t s, const double* G, int n2, int m, int k, int q, Key key,
                            uint64_t i, int j, const SiBuffers& b, int* status);

// FP64 symmetric eigendecomposition of A (n x n, destroyed) by one block:
// evals (nev, descending), X (n x nev, ldx).
as_status launch_eig(cudaStream_t s, int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                     double* work);

// FD shrink weights: sign-canonicalise columns j < l-1 of U (n2 x l) and
// write W[j][p] = sqrt(max(lam_j - lam_l, 0) / lam_j) * u_j[p] (FP32, (l-1) x n2).
as_status launch_shrink_weights(cudaStream_t s, int n2, int ell, const double* lam, double* U, float* W);

// Query helpers.
as_status launch_shrink_rows(cudaStream_t s, int d, int ell, const double* lam, const double* V, int ldv,
                             float* out, long long ldo);

}  // namespace as
