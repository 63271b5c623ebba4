// FP64 symmetric eigensolver spread over the whole GPU, for the large core
// matrices (the 2l x 2l Gram of the FD shrink when l is large, and the query).
// Same method as eig.cuh (Householder tridiagonalisation, Sturm bisection,
// inverse iteration, back-transformation), with each phase split across
// thread blocks:
//   * tridiagonalisation step k: kernel 1 forms v_k (every block recomputes it
//     from row k) and p = A22 v_k, one warp per row, with per-block partial
//     sums of v^T p; kernel 2 sums the partials in a fixed order and applies
//     A22 -= v w^T + w v^T, w = 2p - 2(v^T p) v.  No atomics: results are
//     bitwise reproducible.
//   * bisection: one warp per eigenvalue (multisection); inverse iteration:
//     one thread per eigenvalue.
//   * back-transformation: each block owns a slab of eigenvector columns in
//     shared memory and applies every reflector to it.
#include "eig.cuh"
#include "kernels.cuh"

namespace as {

namespace {

constexpr int kTriRowsPerBlock = 8;  // one warp per row of p

struct TriWork {
  double* d;      // n
  double* e;      // n
  double* v;      // n (current Householder vector)
  double* p;      // n
  double* part;   // partial sums of v^T p, one per block of kernel 1
  double* v2;     // n (second buffer of the fused steps)
  double* p2;     // n
  double* part2;  // partials of the second buffer
};

__device__ __forceinline__ void house_params(const double* row, int m, double* red, double& s_out,
                                             double& alpha, double& vn) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += row[i] * row[i];
  s = block_sum(s, red);
  const double x0 = row[0];
  s_out = s;
  if (s == 0.0) { alpha = 0.0; vn = 1.0; return; }
  alpha = (x0 >= 0.0) ? -sqrt(s) : sqrt(s);
  vn = sqrt(s - x0 * x0 + (x0 - alpha) * (x0 - alpha));
}

__global__ void __launch_bounds__(256) tri_step1(double* A, int lda, int n, int k, TriWork w) {
  extern __shared__ double vs[];  // m doubles
  __shared__ double red[32];
  const int m = n - k - 1;
  const double* row = A + (size_t)k * lda + (k + 1);
  double s, alpha, vn;
  house_params(row, m, red, s, alpha, vn);
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    vs[i] = (s == 0.0) ? 0.0 : ((i == 0) ? (row[0] - alpha) : row[i]) / vn;
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) w.v[i] = vs[i];
    if (threadIdx.x == 0) { w.d[k] = A[(size_t)k * lda + k]; w.e[k] = alpha; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * kTriRowsPerBlock + wid;
  double contrib = 0.0;
  if (i < m) {
    const double* ar = A + (size_t)(k + 1 + i) * lda + (k + 1);
    double acc = 0.0;
    for (int j = lane; j < m; j += 32) acc += ar[j] * vs[j];
    acc = warp_sum(acc);
    if (lane == 0) { w.p[i] = acc; contrib = acc * vs[i]; }
  }
  // deterministic block partial of v^T p (warp order)
  __shared__ double wpart[kTriRowsPerBlock];
  if (lane == 0) wpart[wid] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kTriRowsPerBlock; ++q) t += wpart[q];
    w.part[blockIdx.x] = t;
  }
}

// Fused step k (k >= 0): apply step k's update A22 -= v w^T + w v^T
// (w = 2p - 2(v^T p)v) to rows and columns >= k+2, and in the same pass form
// step k+1's Householder vector (every block recomputes it from the updated
// row k+1) and p_{k+1} = A22' v_{k+1}.  Row and column k+1 of A are not
// updated: only their diagonal (d[k+1]) and v_{k+1} are needed afterwards.
// Double-buffered vectors: in = (v_k, p_k, parts_k), out = (v_{k+1}, p_{k+1}, parts_{k+1}),
// indexed by absolute row (entries [k+1, n) of in, [k+2, n) of out).
struct TriVec { double* v; double* p; double* part; int nparts; };

__global__ void __launch_bounds__(256) tri_fused(double* A, int lda, int n, int k, TriVec in, TriVec out,
                                                 double* d, double* e) {
  extern __shared__ double sm[];
  double* wk = sm;          // w_k[j], j in [k+1, n)   (offset k+1)
  double* vk = sm + n;      // v_k[j]
  double* vn_ = sm + 2 * n; // v_{k+1}[j], j in [k+2, n)
  __shared__ double red[32];
  __shared__ double c_s;
  const int tid = threadIdx.x;
  if (tid < 32) {   // v^T p from the previous step's block partials (fixed order)
    double c = 0.0;
    for (int q = tid; q < in.nparts; q += 32) c += in.part[q];
    c = warp_sum(c);
    if (tid == 0) c_s = c;
  }
  __syncthreads();
  const double c = c_s;
  for (int j = k + 1 + tid; j < n; j += blockDim.x) {
    const double v = in.v[j];
    vk[j] = v;
    wk[j] = 2.0 * in.p[j] - 2.0 * c * v;
  }
  __syncthreads();
  const int k1 = k + 1;
  const double vk1 = vk[k1], wk1 = wk[k1];
  if (blockIdx.x == 0) {
    // keep v_k in row k of A for the back-transformation; d[k+1] = updated diagonal
    for (int j = k + 1 + tid; j < n; j += blockDim.x) A[(size_t)k * lda + j] = vk[j];
    if (tid == 0) d[k1] = A[(size_t)k1 * lda + k1] - 2.0 * vk1 * wk1;
  }
  if (k1 + 1 >= n) return;
  // updated row k+1 over columns [k+2, n): x_j = A[k+1][j] - v_{k+1} w_j - w_{k+1} v_j
  const int m1 = n - k1 - 1;
  double s = 0.0;
  for (int j = k1 + 1 + tid; j < n; j += blockDim.x) {
    const double x = A[(size_t)k1 * lda + j] - vk1 * wk[j] - wk1 * vk[j];
    vn_[j] = x;
    s += x * x;
  }
  s = block_sum(s, red);
  if (m1 == 1) {
    // last 2 x 2 block: no further reflector
    if (blockIdx.x == 0 && tid == 0) {
      const int j = n - 1;
      e[k1] = vn_[j];
      d[j] = A[(size_t)j * lda + j] - 2.0 * vk[j] * wk[j];
      e[j] = 0.0;
    }
    return;
  }
  const double x0 = vn_[k1 + 1];
  double alpha = 0.0, vnorm = 1.0;
  if (s > 0.0) {
    alpha = (x0 >= 0.0) ? -sqrt(s) : sqrt(s);
    vnorm = sqrt(s - x0 * x0 + (x0 - alpha) * (x0 - alpha));
  }
  __syncthreads();
  for (int j = k1 + 1 + tid; j < n; j += blockDim.x)
    vn_[j] = (s == 0.0) ? 0.0 : ((j == k1 + 1) ? (vn_[j] - alpha) : vn_[j]) / vnorm;
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int j = k1 + 1 + tid; j < n; j += blockDim.x) out.v[j] = vn_[j];
    if (tid == 0) e[k1] = alpha;
  }
  // rows i in [k+2, n): one warp per row; update and dot with v_{k+1}
  const int lane = tid & 31, wid = tid >> 5;
  const int i = k1 + 1 + blockIdx.x * 8 + wid;
  double contrib = 0.0;
  if (i < n) {
    double* ar = A + (size_t)i * lda;
    const double vi = vk[i], wi = wk[i];
    double acc = 0.0;
    for (int j = k1 + 1 + lane; j < n; j += 32) {
      const double a = ar[j] - vi * wk[j] - wi * vk[j];
      ar[j] = a;
      acc += a * vn_[j];
    }
    acc = warp_sum(acc);
    if (lane == 0) { out.p[i] = acc; contrib = acc * vn_[i]; }
  }
  __shared__ double wpart[8];
  if (lane == 0) wpart[wid] = contrib;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += wpart[q];
    out.part[blockIdx.x] = t;
  }
}

__global__ void tri_tail(const double* A, int lda, int n, TriWork w) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    w.d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
    w.e[n - 2] = A[(size_t)(n - 2) * lda + (n - 1)];
    w.d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    w.e[n - 1] = 0.0;
  }
}

// tnorm, pivmin of T
__global__ void tri_norm(int n, TriWork w, double* out2) {
  __shared__ double red[32];
  double tn = 0.0, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double el = (i > 0) ? fabs(w.e[i - 1]) : 0.0, er = (i + 1 < n) ? fabs(w.e[i]) : 0.0;
    tn = fmax(tn, fabs(w.d[i]) + el + er);
    em = fmax(em, er * er);
  }
  tn = block_max(tn, red);
  em = block_max(em, red);
  if (threadIdx.x == 0) { out2[0] = tn; out2[1] = 2.2250738585072014e-308 * fmax(1.0, em); }
}

// One warp per eigenvalue: multisection on Sturm counts (each round the 32
// lanes evaluate 31 interior points, narrowing the bracket 32-fold) down to an
// absolute width of 4 eps ||T||, then inverse iteration by lane 0.
__global__ void bisect_invit(int n, int nev, TriWork w, const double* norms, double* evals, double* X, int ldx,
                             double* lu) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nev) return;
  const double tnorm = norms[0], pivmin = norms[1];
  const double eps = 2.220446049250313e-16;
  const double* d = w.d;
  const double* e = w.e;
  const int idx = n - 1 - j;
  double lo = -tnorm - 2 * eps * tnorm - pivmin, hi = tnorm + 2 * eps * tnorm + pivmin;
  const double atol = 4 * eps * fmax(tnorm, pivmin);
  for (int it = 0; it < 40; ++it) {
    if (hi - lo <= atol + 2 * eps * fmax(fabs(lo), fabs(hi))) break;
    // lane l evaluates x_l = lo + (l+1) (hi-lo)/32, l = 0..30; lane 31 idle
    const double x = lo + (double)(lane + 1) * ((hi - lo) / 32.0);
    const bool above = (lane < 31) ? (sturm_count(n, d, e, x, pivmin) > idx) : true;
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    const int first = __ffs(mask) - 1;   // smallest lane whose point lies above the eigenvalue
    const double nlo = (first == 0) ? lo : lo + (double)first * ((hi - lo) / 32.0);
    const double nhi = (first >= 31) ? hi : lo + (double)(first + 1) * ((hi - lo) / 32.0);
    if (!(nhi > nlo)) break;
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double lam = (tnorm == 0.0) ? 0.0 : 0.5 * (lo + hi);   // a zero matrix has exact zero eigenvalues
  evals[j] = lam;
  // inverse iteration (same factorisation as eig.cuh)
  const double tiny = fmax(eps * tnorm, 1e-300);
  double* u0 = lu + (size_t)(0 * n) * nev + j;
  double* u1 = lu + (size_t)(1 * n) * nev + j;
  double* u2 = lu + (size_t)(2 * n) * nev + j;
  double* ll = lu + (size_t)(3 * n) * nev + j;
  double* pv = lu + (size_t)(4 * n) * nev + j;
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
    return;
  }
  for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] = ii_start(i, j);
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i + 1 < n; ++i) {
      double yi = X[(size_t)i * ldx + j], yn = X[(size_t)(i + 1) * ldx + j];
      if (pv[(size_t)i * nev] != 0.0) { const double t = yi; yi = yn; yn = t; }
      yn -= ll[(size_t)i * nev] * yi;
      X[(size_t)i * ldx + j] = yi;
      X[(size_t)(i + 1) * ldx + j] = yn;
    }
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

// Modified Gram-Schmidt inside clusters of close eigenvalues (one block).
__global__ void cluster_mgs(int n, int nev, const double* norms, const double* evals, double* X, int ldx) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double ctol = 1e-9 * fmax(norms[0], norms[1]);
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
}

// Back-transformation: each block owns columns [c0, c0 + kSlab) of X.
constexpr int kSlab = 4;
__global__ void __launch_bounds__(256) back_transform(const double* A, int lda, int n, int nev, double* X, int ldx) {
  extern __shared__ double xs[];  // n x kSlab
  __shared__ double red[kSlab][8];
  const int c0 = blockIdx.x * kSlab;
  const int nc = min(kSlab, nev - c0);
  for (int e = threadIdx.x; e < n * kSlab; e += blockDim.x) {
    const int i = e / kSlab, c = e - i * kSlab;
    xs[e] = (c < nc) ? X[(size_t)i * ldx + c0 + c] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const double* v = A + (size_t)k * lda + (k + 1);
    double s[kSlab];
#pragma unroll
    for (int c = 0; c < kSlab; ++c) s[c] = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double vi = v[i];
#pragma unroll
      for (int c = 0; c < kSlab; ++c) s[c] += vi * xs[(k + 1 + i) * kSlab + c];
    }
#pragma unroll
    for (int c = 0; c < kSlab; ++c) {
      const double t = warp_sum(s[c]);
      if (lane == 0) red[c][wid] = t;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kSlab; ++c) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += red[c][q];
      s[c] = 2.0 * t;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double vi = v[i];
#pragma unroll
      for (int c = 0; c < kSlab; ++c) xs[(k + 1 + i) * kSlab + c] -= s[c] * vi;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * kSlab; e += blockDim.x) {
    const int i = e / kSlab, c = e - i * kSlab;
    if (c < nc) X[(size_t)i * ldx + c0 + c] = xs[e];
  }
}

}  // namespace

size_t eig_large_work_doubles(int n, int nev) {
  const int nparts = (n + kTriRowsPerBlock - 1) / kTriRowsPerBlock;
  return 6 * (size_t)n + 2 * (size_t)nparts + 2 + 5 * (size_t)n * nev + 64;
}

as_status launch_eig_large(cudaStream_t s, int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                           double* work, Prof* prof) {
  if (n < 3) return launch_eig(s, n, A, lda, nev, evals, X, ldx, work);
  TriWork w;
  w.d = work;
  w.e = w.d + n;
  w.v = w.e + n;
  w.p = w.v + n;
  w.part = w.p + n;
  const int nparts_max = (n + kTriRowsPerBlock - 1) / kTriRowsPerBlock;
  w.v2 = w.part + nparts_max;
  w.p2 = w.v2 + n;
  w.part2 = w.p2 + n;
  double* norms = w.part2 + nparts_max;
  double* lu = norms + 2;
  const size_t smem1 = (size_t)n * sizeof(double);
  AS_CUDA_TRY(cudaFuncSetAttribute(tri_step1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
  if (prof) prof->begin(PK_EIG_TRI, s);
  {
    // step 0 forms v_0 and p_0 = A22 v_0 (written to absolute rows 1..n-1)
    const int m = n - 1;
    const int nb = (m + kTriRowsPerBlock - 1) / kTriRowsPerBlock;
    tri_step1<<<nb, 256, (size_t)m * sizeof(double), s>>>(A, lda, n, 0, w); count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
    TriVec buf[2];
    buf[0] = TriVec{w.v - 1, w.p - 1, w.part, nb};   // v_0, p_0 indexed by absolute row
    buf[1] = TriVec{w.v2, w.p2, w.part2, 0};
    const size_t smem = 3 * (size_t)n * sizeof(double);
    // opt in for the dynamic size itself: the static shared memory comes on top
    AS_CUDA_TRY(cudaFuncSetAttribute(tri_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int k = 0; k + 2 < n; ++k) {
      TriVec& in = buf[k & 1];
      TriVec& out = buf[(k + 1) & 1];
      const int rows = n - k - 2;           // rows k+2..n-1
      const int grid = std::max(1, (rows + 7) / 8);
      out.nparts = grid;
      tri_fused<<<grid, 256, smem, s>>>(A, lda, n, k, in, out, w.d, w.e); count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
      // the buffers alternate; the base pointers of buffer 0 are re-pointed to
      // absolute indexing after the first step
      if (k == 0) buf[0] = TriVec{w.v, w.p, w.part, 0};
    }
  }
  if (prof) prof->end(PK_EIG_TRI, s, 4.0 / 3.0 * (double)n * n * n, 8.0 * (double)n * n);
  if (prof) prof->begin(PK_EIG_SOLVE, s);
  tri_norm<<<1, 256, 0, s>>>(n, w, norms); count_launches(1);
  bisect_invit<<<(nev + 3) / 4, 128, 0, s>>>(n, nev, w, norms, evals, X, ldx, lu); count_launches(1);
  cluster_mgs<<<1, 512, 0, s>>>(n, nev, norms, evals, X, ldx); count_launches(1);
  if (prof) prof->end(PK_EIG_SOLVE, s, 0.0, 0.0);
  if (prof) prof->begin(PK_EIG_BACK, s);
  const size_t smem3 = (size_t)n * kSlab * sizeof(double);
  AS_CUDA_TRY(cudaFuncSetAttribute(back_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3));
  back_transform<<<(nev + kSlab - 1) / kSlab, 256, smem3, s>>>(A, lda, n, nev, X, ldx); count_launches(1);
  if (prof) prof->end(PK_EIG_BACK, s, 2.0 * (double)n * n * nev, 8.0 * (double)n * n);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
