// Symmetric eigensolver spread over the whole GPU, for the large core
// matrices (the 2l x 2l Gram of the FD shrink when l is large, and the query).
// FP64 in and out.  Method: Householder tridiagonalisation, Sturm bisection,
// inverse iteration, back-transformation (as eig.cuh).  The O(n^3) loops run
// in double-float arithmetic (df64.cuh, about 48 significant bits) on the
// FP32 pipes, because FP64 throughput is a small fraction of FP32 on this
// part; A is scaled by a power of two so that its entries fit FP32's
// exponent range, and converted in place.
//   * tridiagonalisation (df64): one cooperative launch, one grid barrier per
//     column; pass r applies update r-1 (A22 -= v w^T + w v^T,
//     w = 2p - 2(v^T p) v) and, in the same sweep over the rows, forms v_r
//     (every block recomputes it from row r) and p = A22 v_r, one warp per
//     row, with per-block partial sums of v^T p summed in a fixed order by the
//     next pass.  No atomics: results are bitwise reproducible.
//   * bisection: several lanes per eigenvalue (multisection, the lane count
//     picked per matrix order by the launch-shape autotuner) on df64 Sturm
//     counts of T / ||T||; inverse iteration in df64 on T / ||T||, one
//     thread per eigenvalue, its tridiagonal factors staged through shared
//     memory with cp.async (FP64 for the rare eigenvector whose df64 iterate
//     leaves the FP32 range).
//   * back-transformation (df64, blocked): reflectors are grouped into
//     compact-WY factors I - V T V^T; each block owns a slab of eigenvector
//     columns in shared memory and applies the groups to it.
#include "df64.cuh"
#include "eig.cuh"
#include "grid.cuh"
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

// Lanes per eigenvalue of the multisection: LANES - 1 interior points per
// round narrow the bracket LANES-fold.  More lanes mean fewer dependent
// rounds but more Sturm counts per bit; the launcher lets the autotuner pick
// 4, 8, 16 or 32 per matrix order (8 when tuning is off).

// Modified Gram-Schmidt inside clusters of close eigenvalues (one block).
__global__ void cluster_mgs(int n, int nev, const double* norms, const double* evals, double* X, int ldx) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double ctol = 1e-9 * fmax(norms[0], norms[1]) * norms[3];   // evals are unscaled
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



// ---- double-float (df64) kernels -------------------------------------------
// T scaled by 1/||T|| in df64: dd[i] = d_i / tn, ee[i] = e_i / tn and
// e2[i] = (e_i / tn)^2.  With |entries| <= 1 the Sturm recurrence and the
// inverse iteration stay far from FP32 overflow.
__global__ void tri_scale_df(int n, TriWork w, const double* norms, df64* dd, df64* e2, df64* ee) {
  const double tn = norms[0];
  const double inv = (tn > 0.0) ? 1.0 / tn : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dd[i] = df_from_double(w.d[i] * inv);
    const double es = (i + 1 < n) ? w.e[i] * inv : 0.0;
    ee[i] = df_from_double(es);
    e2[i] = df_from_double(es * es);
  }
}

// a / b from one FP32 reciprocal of b.hi: q1 = a.hi / b.hi and the
// correction (a - q1 b) / b.hi, both through the same reciprocal; accurate to
// about 2^-44 relative (one special-function instruction per quotient).
__device__ __forceinline__ df64 df_div_fast(df64 a, df64 b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, rb);
  float p, e;
  two_prod(q1, b.hi, p, e);
  float s, f;
  two_sum(a.hi, -p, s, f);
  f = __fsub_rn(f, e);
  f = __fadd_rn(f, a.lo);
  f = __fmaf_rn(-q1, b.lo, f);
  const float q2 = __fmul_rn(__fadd_rn(s, f), rb);
  return df_renorm(q1, q2);
}

// Number of eigenvalues of the scaled T below x (LDL^T pivots in df64; a
// pivot smaller than pivmin is replaced by -pivmin as in the FP64 count).
__device__ int sturm_count_df(int n, const df64* dd, const df64* e2, df64 x, float pivmin) {
  int c = 0;
  df64 q = df_sub(dd[0], x);
  if (fabsf(q.hi) < pivmin) q = df64{-pivmin, 0.f};
  if (q.hi < 0.f) ++c;
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    q = df_sub(df_sub(dd[i], x), df_div_fast(e2[i - 1], q));
    if (fabsf(q.hi) < pivmin) q = df64{-pivmin, 0.f};
    if (q.hi < 0.f) ++c;
  }
  return c;
}

// Multisection on the scaled T with df64 Sturm counts (kBisLanes lanes per
// eigenvalue), then inverse iteration in FP64 by the group's first lane.  The
// bracket is kept in FP64; evaluation points are rounded to df64.  Stops at a
// width of 2^-44 of ||T|| (df64 resolution).
template <int kBisLanes>
__global__ void bisect_df(int n, int nev, const double* norms, const df64* dd, const df64* e2, double* evals) {
  const int lane = threadIdx.x & 31;
  const int g = lane & (kBisLanes - 1), grp = lane / kBisLanes;
  const int j = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / kBisLanes) + grp;
  const bool active = j < nev;
  const double tnorm = norms[0];
  const int idx = n - 1 - j;
  const float pivmin = 0x1p-100f;
  const double tol = 0x1p-44;
  double lo = -1.0 - tol, hi = 1.0 + tol;
  bool stop = !active || tnorm == 0.0;
  for (int it = 0; it < 64; ++it) {
    if (!stop && hi - lo <= tol * fmax(1.0, fmax(fabs(lo), fabs(hi)))) stop = true;
    if (__all_sync(0xffffffffu, stop)) break;
    const double step = (hi - lo) / (double)kBisLanes;
    bool above = true;
    if (!stop && g < kBisLanes - 1)
      above = sturm_count_df(n, dd, e2, df_from_double(lo + (double)(g + 1) * step), pivmin) > idx;
    const unsigned gmask = (kBisLanes == 32) ? 0xffffffffu : ((1u << (kBisLanes & 31)) - 1u);
    const unsigned mask = (__ballot_sync(0xffffffffu, above) >> ((grp * kBisLanes) & 31)) & gmask;
    if (!stop) {
      const int first = __ffs(mask) - 1;
      const double nlo = (first == 0) ? lo : lo + (double)first * step;
      const double nhi = (first >= kBisLanes - 1) ? hi : lo + (double)(first + 1) * step;
      if (!(nhi > nlo)) {
        stop = true;
      } else {
        lo = nlo;
        hi = nhi;
      }
    }
  }
  if (g != 0 || !active) return;
  const double lam = (tnorm == 0.0) ? 0.0 : 0.5 * (lo + hi) * tnorm;   // of the scaled matrix
  evals[j] = lam * norms[3];                                            // exact power-of-two unscaling
}

// Inverse iteration in FP64 for the eigenvalues found by bisect_df (the
// fallback of invit_dd below, for the eigenvectors `only` flags), one thread
// per eigenvector, up to 32 eigenvectors per block: the LU factorisation and the solves
// are FP64 recurrences, and FP64 issue is scarce on this part, so no lane of a
// warp should idle.  lam = evals[j] / norms[3] undoes the exact power-of-two
// unscaling.
//
// The sweeps over the factors are bound by memory latency, not arithmetic:
// their loads do not depend on the recurrence.  The factors and the iterate
// are interleaved by eigenvector (entry i of vector j at i * nev + j), so the
// block's vectors' entries of one step are contiguous (256 bytes for 32); each
// thread copies its own entries of the next kInvitTile steps to shared memory
// with cp.async while it runs the recurrence over the current tile (double
// buffered).  A thread reads back only what it copied itself, so no block
// barrier is needed.  The LU stores the reciprocal of each pivot (off the
// recurrence's dependent chain); the normalisation of an iterate is folded
// into the next forward sweep (the sweep is linear), so an iteration is two
// sweeps; the first iteration starts from ii_start, and one final pass scales
// the last iterate.
constexpr int kInvitTile = 24;   // 2 x 4 x 24 x 32 doubles = 48 KB of static shared memory
constexpr int kInvitArrays = 4;   // staged arrays per step (at most)

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(32) invit_df(int n, int nev, TriWork w, const double* norms, const double* evals,
                                               double* X, int ldx, double* lu, const int* only) {
  // [buffer][array][step][lane]
  __shared__ double stg[2][kInvitArrays][kInvitTile][32];
  const int lane = threadIdx.x;
  // the block is one (possibly partial) warp: name only its threads
  const unsigned wmask = (blockDim.x >= 32) ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const int j = blockIdx.x * blockDim.x + lane;
  // with `only`, just the eigenvectors it flags (the others' lanes compute
  // and store nothing)
  const bool valid = j < nev && (!only || only[j] != 0);
  if (only && __all_sync(wmask, !valid)) return;
  const int jj = (j < nev) ? j : nev - 1;   // an in-range column for the copies of lanes past nev
  const double tnorm = norms[0];
  const double eps = 2.220446049250313e-16;
  const double lam = (tnorm == 0.0) ? 0.0 : evals[jj] / norms[3];
  const double* d = w.d;
  const double* e = w.e;
  if (tnorm == 0.0) {   // zero matrix: any orthonormal basis is an eigenbasis
    if (valid)
      for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] = (i == j) ? 1.0 : 0.0;
    return;
  }
  const double tiny = fmax(eps * tnorm, 1e-300);
  double* u0 = lu + (size_t)(0 * n) * nev + jj;   // 1 / pivot (kept away from zero)
  double* u1 = lu + (size_t)(1 * n) * nev + jj;
  double* u2 = lu + (size_t)(2 * n) * nev + jj;
  double* ll = lu + (size_t)(3 * n) * nev + jj;
  double* pv = lu + (size_t)(4 * n) * nev + jj;
  // LU of T - lam I with partial pivoting (as eig.cuh); lanes past nev
  // repeat the last vector's factorisation and store nothing
  double cd = d[0] - lam, cs = e[0];
  for (int i = 0; i + 1 < n; ++i) {
    const double b = e[i];
    const double nd = d[i + 1] - lam, ns = (i + 2 < n) ? e[i + 1] : 0.0;
    double piv, U1, U2, L, P;
    if (fabs(cd) >= fabs(b)) {
      if (cd == 0.0) cd = tiny;
      const double li = b / cd;
      piv = cd; U1 = cs; U2 = 0.0; L = li; P = 0.0;
      cd = nd - li * cs; cs = ns;
    } else {
      const double li = cd / b;
      piv = b; U1 = nd; U2 = ns; L = li; P = 1.0;
      cd = cs - li * nd; cs = -li * ns;
    }
    if (fabs(piv) < tiny) piv = (piv < 0 ? -tiny : tiny);
    if (valid) {
      u0[(size_t)i * nev] = 1.0 / piv;
      u1[(size_t)i * nev] = U1; u2[(size_t)i * nev] = U2;
      ll[(size_t)i * nev] = L; pv[(size_t)i * nev] = P;
    }
  }
  if (fabs(cd) < tiny) cd = (cd < 0 ? -tiny : tiny);
  if (valid) u0[(size_t)(n - 1) * nev] = 1.0 / cd;
  __threadfence_block();   // the factors (and later the iterate) are read back through cp.async
  __syncwarp(wmask);
  double* x = X + jj;
  const size_t sx = (size_t)ldx;
  double rhs = 1.0;   // scale of the stored iterate (its pending normalisation)
  for (int it = 0; it < 3; ++it) {
    // forward elimination with the row interchanges: y = L^-1 P (rhs x), steps
    // i = 0 .. n-2 in tiles; a tile stages ll[i], pv[i] and x[i+1]
    const int nsteps = n - 1;
    const int ntiles = (nsteps + kInvitTile - 1) / kInvitTile;
    auto stage_fwd = [&](int t, int buf) {
      const int i0 = t * kInvitTile, cnt = min(kInvitTile, nsteps - i0);
      for (int u = 0; u < cnt; ++u) {
        const size_t i = (size_t)(i0 + u);
        cp_async8(&stg[buf][0][u][lane], ll + i * nev);
        cp_async8(&stg[buf][1][u][lane], pv + i * nev);
        if (it > 0) cp_async8(&stg[buf][2][u][lane], x + (i + 1) * sx);
      }
      cp_async_commit();
    };
    double cur = (it == 0) ? ii_start(0, jj) : x[0] * rhs;
    if (ntiles > 0) stage_fwd(0, 0);
    for (int t = 0; t < ntiles; ++t) {
      if (t + 1 < ntiles) {
        stage_fwd(t + 1, (t + 1) & 1);
        cp_async_wait1();
      } else {
        cp_async_wait0();
      }
      const int buf = t & 1, i0 = t * kInvitTile, cnt = min(kInvitTile, nsteps - i0);
      for (int u = 0; u < cnt; ++u) {
        const int i = i0 + u;
        double yi = cur;
        double yn = (it == 0) ? ii_start(i + 1, jj) : stg[buf][2][u][lane] * rhs;
        if (stg[buf][1][u][lane] != 0.0) { const double tt = yi; yi = yn; yn = tt; }
        yn -= stg[buf][0][u][lane] * yi;
        if (valid) x[(size_t)i * sx] = yi;
        cur = yn;
      }
    }
    if (valid) x[(size_t)(n - 1) * sx] = cur;
    __threadfence_block();
    __syncwarp(wmask);
    // back substitution (u0 holds 1 / pivot), with the max and the sum of
    // squares; steps i = n-1 .. 0 in tiles, staging x[i], u0[i], u1[i], u2[i]
    const int btiles = (n + kInvitTile - 1) / kInvitTile;
    auto stage_back = [&](int t, int buf) {
      const int ihi = n - 1 - t * kInvitTile, cnt = min(kInvitTile, ihi + 1);
      for (int u = 0; u < cnt; ++u) {
        const size_t i = (size_t)(ihi - u);
        cp_async8(&stg[buf][0][u][lane], x + i * sx);
        cp_async8(&stg[buf][1][u][lane], u0 + i * nev);
        cp_async8(&stg[buf][2][u][lane], u1 + i * nev);
        cp_async8(&stg[buf][3][u][lane], u2 + i * nev);
      }
      cp_async_commit();
    };
    double xn1 = 0.0, xn2 = 0.0, mx = 0.0, ss = 0.0;
    stage_back(0, 0);
    for (int t = 0; t < btiles; ++t) {
      if (t + 1 < btiles) {
        stage_back(t + 1, (t + 1) & 1);
        cp_async_wait1();
      } else {
        cp_async_wait0();
      }
      const int buf = t & 1, ihi = n - 1 - t * kInvitTile, cnt = min(kInvitTile, ihi + 1);
      for (int u = 0; u < cnt; ++u) {
        const double xi = (stg[buf][0][u][lane] - stg[buf][2][u][lane] * xn1 - stg[buf][3][u][lane] * xn2) *
                          stg[buf][1][u][lane];
        if (valid) x[(size_t)(ihi - u) * sx] = xi;
        xn2 = xn1; xn1 = xi;
        mx = fmax(mx, fabs(xi));
        ss = fma(xi, xi, ss);
      }
    }
    __threadfence_block();
    __syncwarp(wmask);
    if (ss > 0.0 && ss < 1e300) {
      rhs = 1.0 / sqrt(ss);
    } else {   // squares out of range: normalise in two scaled passes
      const double rmx = (mx > 0.0) ? 1.0 / mx : 0.0;
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) { const double v = x[(size_t)i * sx] * rmx; nrm += v * v; }
      rhs = (nrm > 0.0) ? rmx / sqrt(nrm) : 0.0;
    }
  }
  if (valid)
    for (int i = 0; i < n; ++i) x[(size_t)i * sx] *= rhs;
}

// The same inverse iteration in df64 on the FP32 pipes, on T / ||T|| (dd, ee):
// the FP64 recurrences of invit_df are long dependent chains of slow FP64
// instructions on this part.  Same factorisation (partial pivoting, pivots
// kept at least eps in magnitude), the same start ii_start, the same storage
// (a df64 value in each 8-byte slot of lu and X), the same staging, and two
// iterations (kInvitDdIters) instead of three.  The sum of squares is
// accumulated in df64 (compensated) and the reciprocal norm taken with
// df_rsqrt.  An iterate that leaves the FP32 range (several nearly
// zero pivots on one eigenvector) is flagged in bad[j] and left for invit_df,
// which the launcher runs on the flagged eigenvectors afterwards.
// Two iterations: with eigenvalues bisected to 2^-44 of ||T||, the error of an
// eigenvector after two solves is of order (2^-44 / gap)^2, below the 1e-8
// orthogonality of the solver's tests down to the gap at which cluster_mgs
// takes over (1e-9 relative); the FP64 fallback keeps three.
constexpr int kInvitDdIters = 2;

__global__ void __launch_bounds__(32) invit_dd(int n, int nev, const df64* dd, const df64* ee, const double* norms,
                                               const double* evals, double* X, int ldx, double* lu, int* bad) {
  __shared__ df64 stg[2][kInvitArrays][kInvitTile][32];
  const int lane = threadIdx.x;
  const unsigned wmask = (blockDim.x >= 32) ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const int j = blockIdx.x * blockDim.x + lane;
  const bool valid = j < nev;
  const int jj = valid ? j : nev - 1;
  const double tnorm = norms[0];
  if (tnorm == 0.0) {   // zero matrix: any orthonormal basis is an eigenbasis
    if (valid) {
      for (int i = 0; i < n; ++i) X[(size_t)i * ldx + j] = (i == j) ? 1.0 : 0.0;
      bad[j] = 0;
    }
    return;
  }
  const df64 lam = df_from_double(evals[jj] / norms[3] / tnorm);
  const float tiny = 2.220446049250313e-16f;   // eps * ||T / ||T|| ||
  df64* u0 = reinterpret_cast<df64*>(lu) + (size_t)(0 * n) * nev + jj;   // 1 / pivot
  df64* u1 = reinterpret_cast<df64*>(lu) + (size_t)(1 * n) * nev + jj;
  df64* u2 = reinterpret_cast<df64*>(lu) + (size_t)(2 * n) * nev + jj;
  df64* ll = reinterpret_cast<df64*>(lu) + (size_t)(3 * n) * nev + jj;
  df64* pv = reinterpret_cast<df64*>(lu) + (size_t)(4 * n) * nev + jj;
  const df64 zero{0.f, 0.f}, one{1.f, 0.f};
  df64 cd = df_sub(dd[0], lam), cs = ee[0];
  for (int i = 0; i + 1 < n; ++i) {
    const df64 b = ee[i];
    const df64 nd = df_sub(dd[i + 1], lam), ns = (i + 2 < n) ? ee[i + 1] : zero;
    df64 piv, U1, U2, L, P;
    if (fabsf(cd.hi) >= fabsf(b.hi)) {
      if (cd.hi == 0.f) cd = df64{tiny, 0.f};
      const df64 li = df_div_fast(b, cd);
      piv = cd; U1 = cs; U2 = zero; L = li; P = zero;
      cd = df_sub(nd, df_mul(li, cs));
      cs = ns;
    } else {
      const df64 li = df_div_fast(cd, b);
      piv = b; U1 = nd; U2 = ns; L = li; P = one;
      cd = df_sub(cs, df_mul(li, nd));
      cs = df_neg(df_mul(li, ns));
    }
    if (fabsf(piv.hi) < tiny) piv = df64{piv.hi < 0.f ? -tiny : tiny, 0.f};
    if (valid) {
      u0[(size_t)i * nev] = df_div_fast(one, piv);
      u1[(size_t)i * nev] = U1; u2[(size_t)i * nev] = U2;
      ll[(size_t)i * nev] = L; pv[(size_t)i * nev] = P;
    }
  }
  if (fabsf(cd.hi) < tiny) cd = df64{cd.hi < 0.f ? -tiny : tiny, 0.f};
  if (valid) u0[(size_t)(n - 1) * nev] = df_div_fast(one, cd);
  __threadfence_block();
  __syncwarp(wmask);
  df64* x = reinterpret_cast<df64*>(X) + jj;
  const size_t sx = (size_t)ldx;
  df64 rhs = one;
  bool finite = true;
  for (int it = 0; it < kInvitDdIters; ++it) {
    const int nsteps = n - 1;
    const int ntiles = (nsteps + kInvitTile - 1) / kInvitTile;
    auto stage_fwd = [&](int t, int buf) {
      const int i0 = t * kInvitTile, cnt = min(kInvitTile, nsteps - i0);
      for (int u = 0; u < cnt; ++u) {
        const size_t i = (size_t)(i0 + u);
        cp_async8(reinterpret_cast<double*>(&stg[buf][0][u][lane]), reinterpret_cast<const double*>(ll + i * nev));
        cp_async8(reinterpret_cast<double*>(&stg[buf][1][u][lane]), reinterpret_cast<const double*>(pv + i * nev));
        if (it > 0)
          cp_async8(reinterpret_cast<double*>(&stg[buf][2][u][lane]), reinterpret_cast<const double*>(x + (i + 1) * sx));
      }
      cp_async_commit();
    };
    df64 cur = (it == 0) ? df_from_double(ii_start(0, jj)) : df_mul(x[0], rhs);
    if (ntiles > 0) stage_fwd(0, 0);
    for (int t = 0; t < ntiles; ++t) {
      if (t + 1 < ntiles) {
        stage_fwd(t + 1, (t + 1) & 1);
        cp_async_wait1();
      } else {
        cp_async_wait0();
      }
      const int buf = t & 1, i0 = t * kInvitTile, cnt = min(kInvitTile, nsteps - i0);
      for (int u = 0; u < cnt; ++u) {
        const int i = i0 + u;
        df64 yi = cur;
        df64 yn = (it == 0) ? df_from_double(ii_start(i + 1, jj)) : df_mul(stg[buf][2][u][lane], rhs);
        if (stg[buf][1][u][lane].hi != 0.f) { const df64 tt = yi; yi = yn; yn = tt; }
        yn = df_sub(yn, df_mul(stg[buf][0][u][lane], yi));
        if (valid) x[(size_t)i * sx] = yi;
        cur = yn;
      }
    }
    if (valid) x[(size_t)(n - 1) * sx] = cur;
    __threadfence_block();
    __syncwarp(wmask);
    const int btiles = (n + kInvitTile - 1) / kInvitTile;
    auto stage_back = [&](int t, int buf) {
      const int ihi = n - 1 - t * kInvitTile, cnt = min(kInvitTile, ihi + 1);
      for (int u = 0; u < cnt; ++u) {
        const size_t i = (size_t)(ihi - u);
        cp_async8(reinterpret_cast<double*>(&stg[buf][0][u][lane]), reinterpret_cast<const double*>(x + i * sx));
        cp_async8(reinterpret_cast<double*>(&stg[buf][1][u][lane]), reinterpret_cast<const double*>(u0 + i * nev));
        cp_async8(reinterpret_cast<double*>(&stg[buf][2][u][lane]), reinterpret_cast<const double*>(u1 + i * nev));
        cp_async8(reinterpret_cast<double*>(&stg[buf][3][u][lane]), reinterpret_cast<const double*>(u2 + i * nev));
      }
      cp_async_commit();
    };
    df64 xn1 = zero, xn2 = zero;
    float mx = 0.f, ss = 0.f, se = 0.f;
    bool nan = false;
    stage_back(0, 0);
    for (int t = 0; t < btiles; ++t) {
      if (t + 1 < btiles) {
        stage_back(t + 1, (t + 1) & 1);
        cp_async_wait1();
      } else {
        cp_async_wait0();
      }
      const int buf = t & 1, ihi = n - 1 - t * kInvitTile, cnt = min(kInvitTile, ihi + 1);
      for (int u = 0; u < cnt; ++u) {
        const df64 xi = df_mul(df_rank2(stg[buf][0][u][lane], stg[buf][2][u][lane], xn1, stg[buf][3][u][lane], xn2),
                               stg[buf][1][u][lane]);
        if (valid) x[(size_t)(ihi - u) * sx] = xi;
        xn2 = xn1; xn1 = xi;
        mx = fmaxf(mx, fabsf(xi.hi));
        nan = nan || (xi.hi != xi.hi);
        df_dot_step(xi, xi, ss, se);
      }
    }
    __threadfence_block();
    __syncwarp(wmask);
    if (nan || !(mx <= 3.0e38f)) {   // the iterate left the FP32 range (or is not a number)
      finite = false;
      break;
    }
    const df64 sq = df_dot_finish(ss, se);
    if (sq.hi > 0.f && sq.hi <= 3.0e38f) {   // false also when the squares overflowed (NaN)
      rhs = df_rsqrt(sq);
    } else {   // squares out of range: normalise in two scaled passes
      const float rmx = (mx > 0.f) ? 1.f / mx : 0.f;
      float ns = 0.f, ne = 0.f;
      for (int i = 0; i < n; ++i) {
        const df64 v = df_mul(x[(size_t)i * sx], df64{rmx, 0.f});
        df_dot_step(v, v, ns, ne);
      }
      const df64 nrm = df_dot_finish(ns, ne);
      rhs = (nrm.hi > 0.f) ? df_mul(df64{rmx, 0.f}, df_rsqrt(nrm)) : zero;
    }
  }
  if (valid) {
    bad[j] = finite ? 0 : 1;
    double* xd = X + j;
    if (finite)
      for (int i = 0; i < n; ++i) {
        const df64 v = df_mul(x[(size_t)i * sx], rhs);
        xd[(size_t)i * sx] = (double)v.hi + (double)v.lo;
      }
  }
}

__device__ __forceinline__ df64 df_warp_sum(df64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df64 t{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, t);
  }
  return v;
}

// max |A_ij| as the bit pattern of a non-negative double (ordered like an
// unsigned integer), by atomicMax: the result does not depend on the order.
__global__ void amax_bits(const double* A, int lda, int n, unsigned long long* out) {
  __shared__ double red[32];
  double m = 0.0;
  const size_t tot = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e - i * n;
    m = fmax(m, fabs(A[i * lda + j]));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// scale[0] = 2^-e with max |A| * 2^-e in [1, 2) (1 for a zero matrix),
// scale[1] = 2^e: exact powers of two.
__global__ void pow2_scale(const unsigned long long* bits, double* scale) {
  const double m = __longlong_as_double((long long)*bits);
  const int ex = (m > 0.0 && m < INFINITY) ? ilogb(m) : 0;
  scale[0] = ldexp(1.0, -ex);
  scale[1] = ldexp(1.0, ex);
}

// In-place conversion of A * scale (FP64, n x n, ld lda) to df64: the same
// 8 bytes per entry now hold (hi, lo).  The power-of-two scale keeps the
// entries inside the FP32 exponent range.
__global__ void to_df_inplace(double* A, int lda, int n, const double* scale) {
  const double sc = scale[0];
  const size_t tot = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e - i * n;
    double* p = A + i * lda + j;
    const df64 v = df_from_double(*p * sc);
    *reinterpret_cast<df64*>(p) = v;
  }
}

// v_j = (x_j - alpha [j == 0]) / vn in df64 (zero vector when szero).
__device__ __forceinline__ df64 house_v_df(df64 xj, bool first, bool szero, df64 alpha, df64 rvn) {
  if (szero) return df64{0.f, 0.f};
  const df64 t = first ? df_sub(xj, alpha) : xj;
  return df_mul(t, rvn);
}

// The whole tridiagonalisation in one cooperative launch (df64), one grid
// barrier per column.  Pass r (r = 0 .. n-2):
//   1. r >= 1: c = v_{r-1}^T p_{r-1} from the previous pass's per-CTA partials
//      (fixed order), w = 2 p_{r-1} - 2 c v_{r-1};
//   2. d_r = the diagonal entry of row r after update r-1; CTA 0 keeps v_{r-1}
//      in row r-1 of A for the back-transformation;
//   3. row r past the diagonal after update r-1 (every CTA, from A and the
//      vectors) -> the Householder vector v_r and e_r = alpha; the last pass
//      (r = n-2) only closes the 2 x 2 tail;
//   4. the rows i >= r+1 (columns >= r+1) are updated with
//      A -= v w^T + w v^T, and p_r[i] = A[i] . v_r is formed; per-CTA
//      partials of v_r^T p_r;
//   5. grid barrier.
// v stays in shared memory across passes (every CTA computes it); p and the
// partials are double buffered by pass parity.  Step 4 deals the rows to the
// CTAs round-robin and splits a row over several warps when rows are fewer
// than warps; warp 0 finishes the split dots before the barrier.
struct TriPersist {
  df64* A;
  int lda, n;
  df64* p[2];      // p_r, absolute row index
  df64* q[2];      // per-CTA partials of v_r^T p_r
  double* d;
  double* e;
  unsigned* cnt;   // barrier arrivals (zero at launch)
  int* status;
};

constexpr int kTriPre = 4;      // entries of p and of row r per thread loaded at the top of a pass

// kTriThreads threads per CTA (one CTA per SM), kTriUnroll row entries in
// flight per lane: the launcher lets the launch-shape autotuner pick among a
// few shapes per matrix order (more warps hide more latency; fewer leave
// more registers to each thread's independent entries).
template <int kTriThreads, int kTriUnroll>
__global__ void __launch_bounds__(kTriThreads, 1) tri_persist_df(const TriPersist t) {
  constexpr int kTriWarps = kTriThreads / 32;
  extern __shared__ df64 smp[];
  const int n = t.n, G = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  df64* vcur = smp;           // v_{r-1}[j], j in [r, n)
  df64* vnew = smp + n;       // row r, then v_r[j], j in [r+1, n)
  df64* wk = smp + 2 * n;     // w_{r-1}[j], j in [r, n)
  __shared__ df64 red[kTriWarps];
  __shared__ df64 x0_s;
  __shared__ df64 wpart[kTriWarps];
  __shared__ int s_ok;
  // Every thread owns the entries j = r + tid + kTriThreads u of the pass's
  // vectors (row r, w, v_r) and is the only one to write them before the
  // barrier that publishes v_r to the sweep; the pass has four CTA barriers:
  // after the norm partials of row r, after v_r, and the two around the grid
  // arrival.
  for (int r = 0; r <= n - 2; ++r) {
    const bool upd = r >= 1;
    const df64* arow = t.A + (size_t)r * t.lda;
    // the entries of p_{r-1} and of row r are loaded together with the partial
    // sums below: one L2 round trip (they do not depend on the coefficient)
    df64 pjr[kTriPre], ajr[kTriPre];
    const df64* pin = ((r - 1) & 1) ? t.p[1] : t.p[0];
#pragma unroll
    for (int u = 0; u < kTriPre; ++u) {
      const int j = r + tid + kTriThreads * u;
      pjr[u] = (upd && j < n) ? pin[j] : df64{0.f, 0.f};
      ajr[u] = (j < n) ? arow[j] : df64{0.f, 0.f};
    }
    // p_{r-1}[r] in every thread: each thread forms w_{r-1}[r] itself (the
    // same operations as the thread that stores wk[r]), so no block barrier
    // is needed between w and the update of row r; every other entry of w a
    // thread uses there is one it computed
    const df64 pr = upd ? pin[r] : df64{0.f, 0.f};
    df64 wr{0.f, 0.f};
    if (upd) {
      // c = v^T p from the per-CTA partials: every warp sums them itself, in the
      // same order, so all threads hold the same value without a barrier
      const df64* qin = ((r - 1) & 1) ? t.q[1] : t.q[0];
      df64 c{0.f, 0.f};
      for (int g0 = 0; g0 < G; g0 += 256) {
        df64 qb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int g = g0 + 32 * u + lane;
          qb[u] = (g < G) ? qin[g] : df64{0.f, 0.f};
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) c = df_add(c, qb[u]);
      }
      c = df_warp_sum(c);
      const df64 c2{2.f * c.hi, 2.f * c.lo};
      wr = df_sub(df64{2.f * pr.hi, 2.f * pr.lo}, df_mul(c2, vcur[r]));
#pragma unroll
      for (int u = 0; u < kTriPre; ++u) {
        const int j = r + tid + kTriThreads * u;
        if (j < n) wk[j] = df_sub(df64{2.f * pjr[u].hi, 2.f * pjr[u].lo}, df_mul(c2, vcur[j]));
      }
      for (int j = r + tid + kTriThreads * kTriPre; j < n; j += blockDim.x) {
        const df64 pj = pin[j];
        wk[j] = df_sub(df64{2.f * pj.hi, 2.f * pj.lo}, df_mul(c2, vcur[j]));
      }
    }
    const df64 vr = upd ? vcur[r] : df64{0.f, 0.f};
    if (blockIdx.x == 0) {
      if (upd)
        for (int j = r + tid; j < n; j += blockDim.x) t.A[(size_t)(r - 1) * t.lda + j] = vcur[j];
      if (tid == 0) t.d[r] = df_to_double(upd ? df_rank2(arow[r], vr, wr, wr, vr) : arow[r]);
    }
    df64 acc{0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kTriPre; ++u) {
      const int j = r + tid + kTriThreads * u;
      if (j >= r + 1 && j < n) {
        const df64 x = upd ? df_rank2(ajr[u], vr, wk[j], wr, vcur[j]) : ajr[u];
        vnew[j] = x;
        if (j == r + 1) x0_s = x;
        acc = df_fma(x, x, acc);
      }
    }
    for (int j = r + tid + kTriThreads * kTriPre; j < n; j += blockDim.x) {
      const df64 x = upd ? df_rank2(arow[j], vr, wk[j], wr, vcur[j]) : arow[j];
      vnew[j] = x;
      acc = df_fma(x, x, acc);
    }
    // ||x||^2 over the block: warp sums, one barrier, then every thread adds
    // the warps' sums in the same order
    acc = df_warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncwarp();
    __syncthreads();
    // every warp sums the warps' partials by the same butterfly: identical s
    // in every thread
    const df64 s = df_warp_sum((lane < kTriWarps) ? red[lane] : df64{0.f, 0.f});
    if (r == n - 2) {   // 2 x 2 tail: no further reflector
      if (blockIdx.x == 0 && tid == 0) {
        const int j = n - 1;
        t.e[r] = df_to_double(vnew[j]);
        const df64 ajj = t.A[(size_t)j * t.lda + j];
        t.d[j] = df_to_double(upd ? df_rank2(ajj, vcur[j], wk[j], wk[j], vcur[j]) : ajj);
        t.e[j] = 0.0;
      }
      return;
    }
    // Householder scalars in df64 (FP64 instructions are slow on this part and
    // these sit on every pass's critical path): alpha = -sign(x0) ||x||, and
    // ||x - alpha e_1||^2 = s - x0^2 + (|x0| + ||x||)^2 = 2 (s + |x0| ||x||)
    const df64 x0 = x0_s;
    const bool szero = !(s.hi > 0.f);
    df64 alpha{0.f, 0.f}, rvn{1.f, 0.f};
    if (!szero) {
      const df64 sq = df_mul(s, df_rsqrt(s));
      alpha = (x0.hi >= 0.f) ? df_neg(sq) : sq;
      const df64 ax0 = (x0.hi >= 0.f) ? x0 : df_neg(x0);
      const df64 h = df_add(s, df_mul(ax0, sq));
      rvn = df_rsqrt(df64{2.f * h.hi, 2.f * h.lo});
    }
    // v_r from this thread's own entries of x (x0 came through x0_s)
#pragma unroll
    for (int u = 0; u < kTriPre; ++u) {
      const int j = r + tid + kTriThreads * u;
      if (j >= r + 1 && j < n) vnew[j] = house_v_df(vnew[j], j == r + 1, szero, alpha, rvn);
    }
    for (int j = r + tid + kTriThreads * kTriPre; j < n; j += blockDim.x)
      vnew[j] = house_v_df(vnew[j], j == r + 1, szero, alpha, rvn);
    if (blockIdx.x == 0 && tid == 0) t.e[r] = df_to_double(alpha);
    __syncwarp();
    __syncthreads();
    // rows i = r+1 .. n-1 (k = i - r - 1 < R): update with (v_{r-1}, w_{r-1})
    // and dot with v_r.  Rows are dealt to the CTAs round-robin (row k to CTA
    // k mod G), so that every SM keeps work as the trailing matrix shrinks;
    // when there are fewer rows than warps, S warps share a row (warp sub of
    // the row takes its 32-column chunks sub, sub + S, ...).  Each warp
    // issues the next kTriUnroll chunks' loads before it works on the current
    // ones.
    df64* pout = (r & 1) ? t.p[1] : t.p[0];
    const int R = n - 1 - r;
    int S = 1;
    while (S < kTriWarps && (long long)R * (2 * S) <= (long long)G * kTriWarps) S *= 2;
    const int slots = kTriWarps / S, slot = warp / S, sub = warp - slot * S;
    const int cstride = 32 * S;                 // columns between a warp's chunks
    df64 contrib{0.f, 0.f};                     // S = 1: sum of p_r[i] v_r[i] over this warp's rows
    df64 mydot{0.f, 0.f};                       // S > 1: this warp's part of its one row's dot
    for (int k = blockIdx.x + G * slot; k < R; k += G * slots) {
      const int i = r + 1 + k;
      df64* ar = t.A + (size_t)i * t.lda;
      const df64 vi = upd ? vcur[i] : df64{0.f, 0.f};
      const df64 wi = upd ? wk[i] : df64{0.f, 0.f};
      // the dot with v_r in two compensated accumulators (s, e): s sums the
      // FP32 products of the high parts through TwoSum, e gathers every error
      // and cross term; only one FP32 add per entry is on each loop-carried chain
      float ds0 = 0.f, de0 = 0.f, ds1 = 0.f, de1 = 0.f;
      auto load = [&](df64 (&b)[kTriUnroll], int jb) {
#pragma unroll
        for (int u = 0; u < kTriUnroll; ++u) {
          const int j = jb + cstride * u;
          b[u] = (j < n) ? ar[j] : df64{0.f, 0.f};
        }
      };
      auto work = [&](df64 (&b)[kTriUnroll], int jb) {
#pragma unroll
        for (int u = 0; u < kTriUnroll; ++u) {
          const int j = jb + cstride * u;
          if (j < n) {
            df64 a = b[u];
            if (upd) {
              a = df_rank2(a, vi, wk[j], wi, vcur[j]);
              ar[j] = a;
            }
            if (u & 1) df_dot_step(a, vnew[j], ds1, de1);
            else df_dot_step(a, vnew[j], ds0, de0);
          }
        }
      };
      // jb - lane is the same in every lane, so the round tests are uniform
      const int rstep = cstride * kTriUnroll;
      df64 b0[kTriUnroll], b1[kTriUnroll];
      int jb = r + 1 + 32 * sub + lane;
      load(b0, jb);
      while (true) {
        bool more = jb + rstep - lane < n;
        if (more) load(b1, jb + rstep);
        work(b0, jb);
        if (!more) break;
        jb += rstep;
        more = jb + rstep - lane < n;
        if (more) load(b0, jb + rstep);
        work(b1, jb);
        if (!more) break;
        jb += rstep;
      }
      df64 dot = df_add(df_dot_finish(ds0, de0), df_dot_finish(ds1, de1));
      dot = df_warp_sum(dot);
      if (S == 1) {
        if (lane == 0) {
          pout[i] = dot;
          contrib = df_add(contrib, df_mul(dot, vnew[i]));
        }
      } else {
        mydot = dot;   // at most one row per warp: R * S <= G * kTriWarps
      }
    }
    if (lane == 0) wpart[warp] = (S == 1) ? contrib : mydot;
    __syncwarp();
    __syncthreads();
    // warp 0 finishes the shared rows' dots (fixed order), forms this CTA's
    // partial of v_r^T p_r, publishes it and arrives at the grid barrier
    df64* qout = (r & 1) ? t.q[1] : t.q[0];
    if (warp == 0) {
      df64 cq{0.f, 0.f};
      if (S == 1) {
        if (lane < kTriWarps) cq = wpart[lane];
      } else if (lane < slots) {
        const int k = blockIdx.x + G * lane;
        if (k < R) {
          df64 dot = wpart[lane * S];
          for (int u = 1; u < S; ++u) dot = df_add(dot, wpart[lane * S + u]);
          const int i = r + 1 + k;
          pout[i] = dot;
          cq = df_mul(dot, vnew[i]);
        }
      }
      cq = df_warp_sum(cq);
      if (lane == 0) qout[blockIdx.x] = cq;
      __syncwarp();
      if (lane == 0) s_ok = grid_arrive_wait(t.cnt, (unsigned)(r + 1) * (unsigned)G, t.status) ? 1 : 0;
    }
    __syncwarp();
    __syncthreads();
    if (!s_ok) return;
    df64* tmp = vcur;   // v_r becomes the vector of the next pass's update
    vcur = vnew;
    vnew = tmp;
  }
}

// Back-transformation in df64, blocked (compact WY).  The reflectors
// H_k = I - 2 v_k v_k^T (k = 0 .. n-3, v_k unit, in row k of the df64 matrix Vd
// at columns k+1 .. n-1) are taken kBtNb at a time: H_k0 ... H_k1-1 =
// I - V T V^T with T upper triangular (T_ii = 2 and
// T[0:i, i] = -2 T[0:i, 0:i] (V[:, 0:i]^T v_i), the forward column recurrence of
// the compact WY form; bt_tfactor_df builds it per group).  Each block of
// bt_apply_df owns SW columns of X (df64 in shared memory) and applies the
// groups from the last to the first: W = V^T X, W <- T W, X <- X - V W: three
// block-wide steps per group instead of two per reflector.
constexpr int kBtNb = 16;

__global__ void __launch_bounds__(256) bt_tfactor_df(const df64* Vd, int ldv, int n, int nk, df64* Tout) {
  const int g = blockIdx.x;
  const int k0 = g * kBtNb, k1 = min(k0 + kBtNb, nk), nbg = k1 - k0;
  __shared__ df64 S[kBtNb][kBtNb];
  __shared__ df64 T[kBtNb][kBtNb];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // S[p][i] = v_{k0+p} . v_{k0+i} (p < i), over rows k0+i+1 .. n-1 where v_{k0+i} lives
  for (int pi = warp; pi < kBtNb * kBtNb; pi += 8) {
    const int p = pi / kBtNb, i = pi - p * kBtNb;
    if (p >= i || i >= nbg) continue;
    const df64* vp = Vd + (size_t)(k0 + p) * ldv;
    const df64* vi = Vd + (size_t)(k0 + i) * ldv;
    df64 a0{0.f, 0.f}, a1{0.f, 0.f};
    int c = k0 + i + 1 + lane;
    for (; c + 32 < n; c += 64) {
      a0 = df_fma(vp[c], vi[c], a0);
      a1 = df_fma(vp[c + 32], vi[c + 32], a1);
    }
    if (c < n) a0 = df_fma(vp[c], vi[c], a0);
    const df64 acc = df_warp_sum(df_add(a0, a1));
    if (lane == 0) S[p][i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < kBtNb; ++i)
      for (int p = 0; p < kBtNb; ++p) T[p][i] = df64{0.f, 0.f};
    for (int i = 0; i < nbg; ++i) {
      T[i][i] = df64{2.f, 0.f};
      for (int p = 0; p < i; ++p) {
        df64 sacc{0.f, 0.f};
        for (int q = p; q < i; ++q) sacc = df_fma(T[p][q], S[q][i], sacc);
        T[p][i] = df64{-2.f * sacc.hi, -2.f * sacc.lo};   // exact scaling by -2
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBtNb * kBtNb; e += blockDim.x)
    Tout[(size_t)g * kBtNb * kBtNb + e] = T[e / kBtNb][e % kBtNb];
}

template <int SW>
__global__ void __launch_bounds__(256) bt_apply_df(const df64* Vd, int ldv, int n, int nk, const df64* Tf, int nev,
                                                    double* X, int ldx) {
  extern __shared__ df64 xd[];  // n x SW
  constexpr int kOut = kBtNb * SW;               // outputs of W
  constexpr int kSplit = 256 / kOut;             // row splits of the W sums
  __shared__ df64 Ts[kBtNb][kBtNb];
  __shared__ df64 Wp[kSplit][kBtNb][SW];
  __shared__ df64 W2[kBtNb][SW];
  const int c0 = blockIdx.x * SW;
  const int nc = min(SW, nev - c0);
  for (int e = threadIdx.x; e < n * SW; e += blockDim.x) {
    const int i = e / SW, c = e - i * SW;
    xd[e] = (c < nc) ? df_from_double(X[(size_t)i * ldx + c0 + c]) : df64{0.f, 0.f};
  }
  const int ngroups = (nk + kBtNb - 1) / kBtNb;
  const int o = threadIdx.x % kOut, sp = threadIdx.x / kOut;
  const int p = o / SW, c = o - p * SW;
  for (int g = ngroups - 1; g >= 0; --g) {
    const int k0 = g * kBtNb, nbg = min(kBtNb, nk - k0);
    for (int e = threadIdx.x; e < kBtNb * kBtNb; e += blockDim.x)
      Ts[e / kBtNb][e % kBtNb] = Tf[(size_t)g * kBtNb * kBtNb + e];
    __syncthreads();   // xd (previous group) and Ts ready
    // W[p][c] = sum over rows i >= k0+p+1 of v_{k0+p}[i] X[i][c], rows split kSplit ways
    {
      df64 a0{0.f, 0.f}, a1{0.f, 0.f};
      if (sp < kSplit && p < nbg) {
        const df64* vp = Vd + (size_t)(k0 + p) * ldv;
        int i = k0 + p + 1 + sp;
        for (; i + kSplit < n; i += 2 * kSplit) {
          a0 = df_fma(vp[i], xd[i * SW + c], a0);
          a1 = df_fma(vp[i + kSplit], xd[(i + kSplit) * SW + c], a1);
        }
        if (i < n) a0 = df_fma(vp[i], xd[i * SW + c], a0);
      }
      if (sp < kSplit) Wp[sp][p][c] = df_add(a0, a1);
    }
    __syncthreads();
    // W2 = T W (T upper triangular), the split partials summed in a fixed order
    if (threadIdx.x < kOut) {
      df64 sacc{0.f, 0.f};
      for (int q = p; q < nbg; ++q) {
        df64 w = Wp[0][q][c];
        for (int t = 1; t < kSplit; ++t) w = df_add(w, Wp[t][q][c]);
        sacc = df_fma(Ts[p][q], w, sacc);
      }
      W2[p][c] = sacc;
    }
    __syncthreads();
    // X[i][c] -= sum_p v_{k0+p}[i] W2[p][c] for rows i >= k0+1 (v_{k0+p}[i] = 0 for i <= k0+p)
    const int rows = n - k0 - 1;
    for (int e = threadIdx.x; e < rows * SW; e += blockDim.x) {
      const int i = k0 + 1 + e / SW, cc = e % SW;
      const int pmax = min(nbg, i - k0);
      df64 s0{0.f, 0.f}, s1{0.f, 0.f};   // two chains: even and odd reflectors
      int q = 0;
      for (; q + 1 < pmax; q += 2) {
        s0 = df_fma(Vd[(size_t)(k0 + q) * ldv + i], W2[q][cc], s0);
        s1 = df_fma(Vd[(size_t)(k0 + q + 1) * ldv + i], W2[q + 1][cc], s1);
      }
      if (q < pmax) s0 = df_fma(Vd[(size_t)(k0 + q) * ldv + i], W2[q][cc], s0);
      xd[i * SW + cc] = df_sub(xd[i * SW + cc], df_add(s0, s1));
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * SW; e += blockDim.x) {
    const int i = e / SW, cc = e - i * SW;
    if (cc < nc) X[(size_t)i * ldx + c0 + cc] = df_to_double(xd[e]);
  }
}

}  // namespace

size_t eig_large_work_doubles(int n, int nev) {
  const int nparts = (n + kTriRowsPerBlock - 1) / kTriRowsPerBlock;
  // ... + the df64 copy of T (2n values, one double each)
  // ... + the barrier counter and a status word (one double)
  // ... + the compact-WY T factors of the back-transformation (kBtNb^2 df64 per group)
  const size_t tf = (size_t)((n + kBtNb - 1) / kBtNb) * kBtNb * kBtNb;
  return 6 * (size_t)n + 2 * (size_t)nparts + 4 + 5 * (size_t)n * nev + 2 * (size_t)n + 1 + 64 + tf;
}

as_status launch_eig_large(cudaStream_t s, int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                           double* work, Prof* prof, int* status) {
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
  double* lu = norms + 4;   // norms: ||T||, pivmin, and the scale of A and its inverse
  df64* dd = reinterpret_cast<df64*>(lu + 5 * (size_t)n * nev);
  df64* e2 = dd + n;
  unsigned* cnt = reinterpret_cast<unsigned*>(e2 + n);
  if (!status) {   // scratch word when the caller passes none, cleared per call
    status = reinterpret_cast<int*>(e2 + n) + 1;
    AS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
  }
  df64* Ad = reinterpret_cast<df64*>(A);
  if (prof) prof->begin(PK_EIG_TRI, s);
  {
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(norms + 2);
    AS_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s));
    amax_bits<<<304, 256, 0, s>>>(A, lda, n, bits); count_launches(1);
    pow2_scale<<<1, 1, 0, s>>>(bits, norms + 2); count_launches(1);
    to_df_inplace<<<1024, 256, 0, s>>>(A, lda, n, norms + 2); count_launches(1);
    // all passes in one cooperative launch (one grid barrier per column)
    int dev = 0, sms = 0;
    AS_CUDA_TRY(cudaGetDevice(&dev));
    AS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(sms, nparts_max));
    const size_t smem = 3 * (size_t)n * sizeof(df64);
    TriPersist tp{};
    tp.A = Ad; tp.lda = lda; tp.n = n;
    tp.p[0] = reinterpret_cast<df64*>(w.p); tp.p[1] = reinterpret_cast<df64*>(w.p2);
    tp.q[0] = reinterpret_cast<df64*>(w.part); tp.q[1] = reinterpret_cast<df64*>(w.part2);
    tp.d = w.d; tp.e = w.e; tp.cnt = cnt; tp.status = status;
    // The reduction overwrites the matrix, so a tuning run starts from a copy
    // of the df64 matrix kept in lu (free until the inverse iteration); when
    // lu is too small for it (few eigenvectors) the default shape runs untuned.
    const size_t abytes = (size_t)n * lda * sizeof(double);
    const bool can_tune = (size_t)lda <= 5 * (size_t)nev;
    bool tuning = false, saved = false;
    auto tri = [&](int shape) -> as_status {
      if (tuning) {
        if (!saved) AS_CUDA_TRY(cudaMemcpyAsync(lu, A, abytes, cudaMemcpyDeviceToDevice, s));
        else AS_CUDA_TRY(cudaMemcpyAsync(A, lu, abytes, cudaMemcpyDeviceToDevice, s));
        saved = true;
      }
      const void* fn = shape == 1 ? (const void*)tri_persist_df<256, 16>
                     : shape == 2 ? (const void*)tri_persist_df<512, 8>
                     : shape == 3 ? (const void*)tri_persist_df<512, 4>
                     : shape == 4 ? (const void*)tri_persist_df<256, 8>
                                  : (const void*)tri_persist_df<512, 16>;
      const int threads = (shape == 1 || shape == 4) ? 256 : 512;
      AS_CUDA_TRY(as_raise_smem_limit(fn, smem));
      int per = 0;
      AS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem));
      if ((long long)per * sms < grid) return AS_ENOTSUP;
      AS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
      void* args[] = {&tp};
      AS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, smem, s));
      count_launches(1);
      return AS_OK;
    };
    // shapes (threads, entries in flight): (512, 16), (256, 16), (512, 8),
    // (512, 4), (256, 8)
    static const int kTriShapes[5] = {0, 1, 2, 3, 4};
    as_status tst = AS_OK;
    bool ran = false;
    tuning = can_tune;   // copies are made only while candidates are timed
    const int shape = can_tune ? tune_pick(s, "tri_persist_df", n, kTriShapes, 5, tri, &tst, &ran) : 0;
    tuning = false;
    if (tst != AS_OK) return tst;
    if (!ran) {   // a cached or default choice, straight on A
      tst = tri(shape);
      if (tst != AS_OK) return tst;
    }
  }
  if (prof) prof->end(PK_EIG_TRI, s, 4.0 / 3.0 * (double)n * n * n, 8.0 * (double)n * n);
  if (prof) prof->begin(PK_EIG_SOLVE, s);
  tri_norm<<<1, 256, 0, s>>>(n, w, norms); count_launches(1);
  tri_scale_df<<<(n + 255) / 256, 256, 0, s>>>(n, w, norms, dd, e2, reinterpret_cast<df64*>(w.v));
  count_launches(1);
  {
    // multisection lanes per eigenvalue, tuned per matrix order
    auto bisect = [&](int lanes) -> as_status {
      const int per_block = (128 / 32) * (32 / lanes);   // eigenvalues per block of 128 threads
      const int nblk = (nev + per_block - 1) / per_block;
      if (lanes == 4) bisect_df<4><<<nblk, 128, 0, s>>>(n, nev, norms, dd, e2, evals);
      else if (lanes == 16) bisect_df<16><<<nblk, 128, 0, s>>>(n, nev, norms, dd, e2, evals);
      else if (lanes == 32) bisect_df<32><<<nblk, 128, 0, s>>>(n, nev, norms, dd, e2, evals);
      else bisect_df<8><<<nblk, 128, 0, s>>>(n, nev, norms, dd, e2, evals);
      count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
      return AS_OK;
    };
    static const int kLaneChoices[4] = {8, 4, 16, 32};
    as_status tst = AS_OK;
    bool ran = false;
    const int lanes = tune_pick(s, "bisect_df", ((long long)n << 20) | (long long)nev, kLaneChoices, 4, bisect,
                                &tst, &ran);
    if (tst != AS_OK) return tst;
    if (!ran) {
      tst = bisect(lanes);
      if (tst != AS_OK) return tst;
    }
    // inverse iteration in df64, eigenvectors per block (one thread each)
    // tuned per matrix order; then the FP64 kernel redoes the eigenvectors
    // whose df64 iterate left the FP32 range (a warp with none returns at once)
    df64* ee = reinterpret_cast<df64*>(w.v);      // free after the reduction
    int* bad = reinterpret_cast<int*>(w.p2);      // n doubles >= nev ints
    auto invit = [&](int per) -> as_status {
      invit_dd<<<(nev + per - 1) / per, per, 0, s>>>(n, nev, dd, ee, norms, evals, X, ldx, lu, bad);
      count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
      return AS_OK;
    };
    static const int kInvitChoices[3] = {32, 16, 8};
    const int per = tune_pick(s, "invit_dd", ((long long)n << 20) | (long long)nev, kInvitChoices, 3, invit, &tst,
                              &ran);
    if (tst != AS_OK) return tst;
    if (!ran) {
      tst = invit(per);
      if (tst != AS_OK) return tst;
    }
    invit_df<<<(nev + 31) / 32, 32, 0, s>>>(n, nev, w, norms, evals, X, ldx, lu, bad);
    count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
  }
  cluster_mgs<<<1, 512, 0, s>>>(n, nev, norms, evals, X, ldx); count_launches(1);
  if (prof) prof->end(PK_EIG_SOLVE, s, 0.0, 0.0);
  if (prof) prof->begin(PK_EIG_BACK, s);
  {
    const int nk = n - 2;   // reflectors k = 0 .. n-3
    const int ngroups = (nk + kBtNb - 1) / kBtNb;
    df64* tf = reinterpret_cast<df64*>(reinterpret_cast<double*>(cnt) + 64);
    bt_tfactor_df<<<ngroups, 256, 0, s>>>(Ad, lda, n, nk, tf); count_launches(1);
    // the widest slab of columns whose df64 copy fits the shared memory and
    // leaves at least three blocks per SM to hide the df64 chains' latency
    int dev = 0, sms = 0;
    AS_CUDA_TRY(cudaGetDevice(&dev));
    AS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int sw0 = 4;
    while (sw0 > 1 && ((size_t)n * sw0 * sizeof(df64) > 160 * 1024 || (nev + sw0 - 1) / sw0 < 3 * sms)) sw0 >>= 1;
    // the slab width is tuned per shape among those whose slab fits 160 KB,
    // the heuristic's choice first; a tuning run starts from a copy of the
    // eigenvectors of T kept in lu (free once the inverse iteration is done)
    const size_t xbytes = (size_t)n * ldx * sizeof(double);
    const bool can_tune_bt = (size_t)ldx <= 5 * (size_t)nev;
    bool bt_tuning = false, bt_saved = false;
    auto bt = [&](int sw) -> as_status {
      if ((size_t)n * sw * sizeof(df64) > 160 * 1024) return AS_ENOTSUP;
      if (bt_tuning) {
        if (!bt_saved) AS_CUDA_TRY(cudaMemcpyAsync(lu, X, xbytes, cudaMemcpyDeviceToDevice, s));
        else AS_CUDA_TRY(cudaMemcpyAsync(X, lu, xbytes, cudaMemcpyDeviceToDevice, s));
        bt_saved = true;
      }
      const size_t smem3 = (size_t)n * sw * sizeof(df64);
      const void* fn = sw == 4 ? (const void*)bt_apply_df<4> : sw == 2 ? (const void*)bt_apply_df<2>
                                                                       : (const void*)bt_apply_df<1>;
      AS_CUDA_TRY(as_raise_smem_limit(fn, smem3));
      const int nb = (nev + sw - 1) / sw;
      if (sw == 4) bt_apply_df<4><<<nb, 256, smem3, s>>>(Ad, lda, n, nk, tf, nev, X, ldx);
      else if (sw == 2) bt_apply_df<2><<<nb, 256, smem3, s>>>(Ad, lda, n, nk, tf, nev, X, ldx);
      else bt_apply_df<1><<<nb, 256, smem3, s>>>(Ad, lda, n, nk, tf, nev, X, ldx);
      count_launches(1);
      AS_CUDA_TRY(cudaGetLastError());
      return AS_OK;
    };
    int swc[3] = {sw0, 0, 0}, nsw = 1;
    for (int c = 4; c >= 1; c >>= 1)
      if (c != sw0) swc[nsw++] = c;
    as_status bst = AS_OK;
    bool bran = false;
    bt_tuning = can_tune_bt;
    const int sw = can_tune_bt ? tune_pick(s, "bt_apply_df", ((long long)n << 20) | (long long)nev, swc, nsw, bt,
                                           &bst, &bran)
                               : sw0;
    bt_tuning = false;
    if (bst != AS_OK) return bst;
    if (!bran) {
      bst = bt(sw);
      if (bst != AS_OK) return bst;
    }
  }
  if (prof) prof->end(PK_EIG_BACK, s, 2.0 * (double)n * n * nev, 8.0 * (double)n * n);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
