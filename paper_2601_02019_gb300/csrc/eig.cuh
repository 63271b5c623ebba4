// FP64 symmetric eigensolver run by one thread block.
//
// Used for the small core factorisations of AeroSketch: the FD shrink's
// eigendecomposition of the 2l x 2l Gram G = C~ C~^T (the SVD of Algorithm 4's
// FD shrink computed through its Gram), the k x k matrices of the Rayleigh-Ritz
// step of Algorithm 2, and the query's eigendecomposition (Algorithm 5).
//
// Method (textbook dense symmetric eigensolver):
//   1. Householder reduction to tridiagonal form, A = Q T Q^T with
//      Q = H_0 H_1 ... H_{n-3}, H_k = I - 2 v_k v_k^T acting on indices > k;
//   2. eigenvalues of T by bisection on Sturm counts, one thread per value;
//   3. eigenvectors of T by inverse iteration with a partially pivoted
//      tridiagonal LU, one thread per vector, then modified Gram-Schmidt
//      inside clusters of close eigenvalues;
//   4. back-transformation u = Q y.
// Only the top `nev` pairs are formed, in descending order.
#pragma once

#include "common.cuh"

namespace as {

struct EigWork {
  // Per-call scratch (global memory), sized by eig_work_doubles(n, nev).
  double* d;     // n      diagonal of T
  double* e;     // n      off-diagonal of T (e[k] couples k and k+1)
  double* lu;    // 5 * n * nev  inverse-iteration factors, interleaved by vector
};

__host__ __device__ inline size_t eig_work_doubles(int n, int nev) {
  return 2 * (size_t)n + 5 * (size_t)n * (size_t)nev + 64;
}

__device__ inline EigWork eig_work_view(double* base, int n, int nev) {
  EigWork w;
  w.d = base;
  w.e = base + n;
  w.lu = base + 2 * (size_t)n;
  return w;
}

// Number of eigenvalues of T (diag d, off-diagonal e) smaller than x.
__device__ inline int sturm_count(int n, const double* d, const double* e, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++c;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
  }
  return c;
}

// Deterministic start vector entries for inverse iteration (not part of the
// method's randomness: any vector with a component along the target works).
__device__ inline double ii_start(int i, int j) {
  uint32_t h = (uint32_t)i * 2654435761u ^ ((uint32_t)j * 2246822519u + 0x9e3779b9u);
  h ^= h >> 15; h *= 2246822519u; h ^= h >> 13; h *= 3266489917u; h ^= h >> 16;
  return ((double)(h & 0xffffff) / 16777216.0) - 0.5 + 1e-3;
}

// A (n x n, row-major, leading dimension lda, generic address space) is
// destroyed: its strict upper triangle receives the Householder vectors.
// evals[0..nev) descending; X column j (X[i*ldx + j]) is the unit eigenvector
// of evals[j].  All threads of the block must call this.
static __device__ void cta_eig_sym(int n, double* A, int lda, int nev, double* evals, double* X,
                            int ldx, EigWork w, double* red /* >= 32 doubles, shared */) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double* d = w.d;
  double* e = w.e;
  if (n == 1) {
    if (tid == 0) { evals[0] = A[0]; X[0] = 1.0; }
    __syncthreads();
    return;
  }
  // 1. tridiagonalisation
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* row = A + (size_t)k * lda + (k + 1);        // x = A[k, k+1:], == A[k+1:, k]
    double s = 0.0;
    for (int i = tid; i < m; i += nt) s += row[i] * row[i];
    s = block_sum(s, red);
    const double x0 = row[0];
    if (tid == 0) d[k] = A[(size_t)k * lda + k];
    if (s == 0.0) {
      if (tid == 0) e[k] = 0.0;
      __syncthreads();
      continue;  // v = 0 stored (row is already zero)
    }
    const double alpha = (x0 >= 0.0) ? -sqrt(s) : sqrt(s);
    const double vn = sqrt(s - x0 * x0 + (x0 - alpha) * (x0 - alpha));
    __syncthreads();
    for (int i = tid; i < m; i += nt) row[i] = (i == 0 ? (x0 - alpha) : row[i]) / vn;  // v
    if (tid == 0) e[k] = alpha;
    __syncthreads();
    // p = A22 v, c = v^T p; store p in column k below the diagonal (A[k+1+i][k])
    double cpart = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double* ar = A + (size_t)(k + 1 + i) * lda + (k + 1);
      double p = 0.0;
      for (int j = 0; j < m; ++j) p += ar[j] * row[j];
      A[(size_t)(k + 1 + i) * lda + k] = p;
      cpart += p * row[i];
    }
    const double c = block_sum(cpart, red);
    // w = 2p - 2cv, kept in column k
    for (int i = tid; i < m; i += nt) {
      double* pi = A + (size_t)(k + 1 + i) * lda + k;
      *pi = 2.0 * (*pi) - 2.0 * c * row[i];
    }
    __syncthreads();
    // A22 -= v w^T + w v^T
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = idx / m, j = idx - i * m;
      const double vi = row[i], vj = row[j];
      const double wi = A[(size_t)(k + 1 + i) * lda + k], wj = A[(size_t)(k + 1 + j) * lda + k];
      A[(size_t)(k + 1 + i) * lda + (k + 1 + j)] -= vi * wj + wi * vj;
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
    e[n - 2] = A[(size_t)(n - 2) * lda + (n - 1)];
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    e[n - 1] = 0.0;
  }
  __syncthreads();

  // 2. bisection
  double tnorm = 0.0, emax2 = 0.0;
  for (int i = tid; i < n; i += nt) {
    const double el = (i > 0) ? fabs(e[i - 1]) : 0.0, er = (i + 1 < n) ? fabs(e[i]) : 0.0;
    tnorm = fmax(tnorm, fabs(d[i]) + el + er);
    emax2 = fmax(emax2, er * er);
  }
  tnorm = block_max(tnorm, red);
  emax2 = block_max(emax2, red);
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  const double eps = 2.220446049250313e-16;
  for (int j = tid; j < nev; j += nt) {
    const int idx = n - 1 - j;  // ascending index of the j-th largest
    double lo = -tnorm - 2 * eps * tnorm - pivmin, hi = tnorm + 2 * eps * tnorm + pivmin;
    for (int it = 0; it < 256; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(n, d, e, mid, pivmin) > idx) hi = mid; else lo = mid;
      if (hi - lo <= 2 * eps * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    }
    evals[j] = (tnorm == 0.0) ? 0.0 : 0.5 * (lo + hi);   // a zero matrix has exact zero eigenvalues
  }
  __syncthreads();

  // 3. inverse iteration, one thread per eigenvalue
  const double tiny = fmax(eps * tnorm, 1e-300);
  for (int j = tid; j < nev; j += nt) {
    const double lam = evals[j];
    double* u0 = w.lu + (size_t)(0 * n) * nev + j;   // entry i at [i * nev]
    double* u1 = w.lu + (size_t)(1 * n) * nev + j;
    double* u2 = w.lu + (size_t)(2 * n) * nev + j;
    double* ll = w.lu + (size_t)(3 * n) * nev + j;
    double* pv = w.lu + (size_t)(4 * n) * nev + j;
    double cd = d[0] - lam, cs = e[0];
    for (int i = 0; i + 1 < n; ++i) {
      const double b = e[i];
      const double nd = d[i + 1] - lam, ns = (i + 2 < n) ? e[i + 1] : 0.0;
      if (fabs(cd) >= fabs(b)) {
        if (cd == 0.0) cd = tiny;
        const double li = b / cd;
        u0[(size_t)i * nev] = cd; u1[(size_t)i * nev] = cs; u2[(size_t)i * nev] = 0.0;
        ll[(size_t)i * nev] = li; pv[(size_t)i * nev] = 0.0;
        cd = nd - li * cs; cs = ns;
      } else {
        const double li = cd / b;
        u0[(size_t)i * nev] = b; u1[(size_t)i * nev] = nd; u2[(size_t)i * nev] = ns;
        ll[(size_t)i * nev] = li; pv[(size_t)i * nev] = 1.0;
        cd = cs - li * nd; cs = -li * ns;
      }
    }
    if (fabs(cd) < tiny) cd = (cd < 0 ? -tiny : tiny);
    u0[(size_t)(n - 1) * nev] = cd;
    for (int i = 0; i < n; ++i) {
      const double p = u0[(size_t)i * nev];
      if (fabs(p) < tiny) u0[(size_t)i * nev] = (p < 0 ? -tiny : tiny);
    }
    if (tnorm == 0.0) {   // zero matrix: any orthonormal basis is an eigenbasis
      for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] = (i == j) ? 1.0 : 0.0;
      continue;
    }
    for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] = ii_start(i, j);
    for (int it = 0; it < 3; ++it) {
      // forward: apply the row interchanges and multipliers
      for (int i = 0; i + 1 < n; ++i) {
        double yi = X[(size_t)i * ldx + j], yn = X[(size_t)(i + 1) * ldx + j];
        if (pv[(size_t)i * nev] != 0.0) { const double t = yi; yi = yn; yn = t; }
        yn -= ll[(size_t)i * nev] * yi;
        X[(size_t)i * ldx + j] = yi;
        X[(size_t)(i + 1) * ldx + j] = yn;
      }
      // back substitution with U (three diagonals)
      double xn1 = 0.0, xn2 = 0.0, mx = 0.0;
      for (int i = n - 1; i >= 0; --i) {
        const double xi = (X[(size_t)i * ldx + j] - u1[(size_t)i * nev] * xn1 - u2[(size_t)i * nev] * xn2) /
                          u0[(size_t)i * nev];
        X[(size_t)i * ldx + j] = xi;
        xn2 = xn1; xn1 = xi;
        mx = fmax(mx, fabs(xi));
      }
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) { const double v = X[(size_t)i * ldx + j] / mx; nrm += v * v; }
      const double sc = 1.0 / (mx * sqrt(nrm));
      for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] *= sc;
    }
  }
  __syncthreads();
  // modified Gram-Schmidt inside clusters of close eigenvalues
  const double ctol = 1e-9 * fmax(tnorm, pivmin);
  int c0 = 0;
  for (int j = 1; j < nev; ++j) {
    if (evals[j - 1] - evals[j] > ctol) { c0 = j; continue; }
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = c0; q < j; ++q) {
        double s = 0.0;
        for (int i = tid; i < n; i += nt) s += X[(size_t)i * ldx + q] * X[(size_t)i * ldx + j];
        s = block_sum(s, red);
        for (int i = tid; i < n; i += nt) X[(size_t)i * ldx + j] -= s * X[(size_t)i * ldx + q];
        __syncthreads();
      }
      double s = 0.0;
      for (int i = tid; i < n; i += nt) s += X[(size_t)i * ldx + j] * X[(size_t)i * ldx + j];
      s = block_sum(s, red);
      const double sc = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
      for (int i = tid; i < n; i += nt) X[(size_t)i * ldx + j] *= sc;
      __syncthreads();
    }
  }
  // 4. back-transformation u = H_0 (H_1 (... (H_{n-3} y)))
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const double* v = A + (size_t)k * lda + (k + 1);
    for (int jj = tid; jj < nev; jj += nt) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += v[i] * X[(size_t)(k + 1 + i) * ldx + jj];
      s *= 2.0;
      for (int i = 0; i < m; ++i) X[(size_t)(k + 1 + i) * ldx + jj] -= s * v[i];
    }
    __syncthreads();
  }
}

}  // namespace as
