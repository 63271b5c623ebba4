// Launchers of the AeroSketch kernels (internal C++ interface of the library).
#pragma once

#include <functional>

#include <cuda.h>
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"

namespace as {

// Optional per-kernel-class event timer (the sketch's AS_PROFILE mode).
enum ProfClass {
  PK_BATCH_GEMM = 0,  // batched G-space iterations (persistent kernel, FP32)
  PK_BATCH_ORTH,      // starting vectors and FP32 mirror of G for the batch
  PK_EIG,             // FP64 eigensolver of the FD shrink
  PK_REBUILD,         // FD rebuild C' = W C~ and G = C' C'^T
  PK_GRAM,            // Gram rows of a block
  PK_INGEST,          // row ingest
  PK_EVENT,           // FP64 single-row path of an event row and the dump
  PK_EIG_TRI,         // eigensolver phase: tridiagonalisation
  PK_EIG_SOLVE,       // eigensolver phase: bisection, inverse iteration, cluster MGS
  PK_EIG_BACK,        // eigensolver phase: back-transformation
  PK_BATCH_TC,        // batched G-space iterations on tcgen05 (tensor forms)
  PK_COUNT
};
// end() records the algorithmic work of the bracketed launches; `issued` is
// the floating-point work they issued when that differs (< 0: the same).  The
// batched iterations compute every row of a block speculatively, so their
// algorithmic work is known only when the block's decisions are taken, and
// add_work() records it then.
struct Prof {
  virtual void begin(int cls, cudaStream_t s) = 0;
  virtual void end(int cls, cudaStream_t s, double flops, double bytes, double issued = -1.0) = 0;
  virtual void add_work(int cls, double flops) = 0;
  virtual ~Prof() {}
};

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
                                 uint64_t i, double* sig2, uint64_t jsub = 0);

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

// Large-matrix FP64 eigensolver spread over the GPU (eig_large.cu); same
// contract as launch_eig.  Work size: eig_large_work_doubles(n, nev).
size_t eig_large_work_doubles(int n, int nev);
// status: sticky status word for a grid-barrier timeout (AS_ETIMEOUT); NULL
// uses a scratch word in `work`, cleared by each call.
as_status launch_eig_large(cudaStream_t s, int n, double* A, int lda, int nev, double* evals, double* X, int ldx,
                           double* work, Prof* prof = nullptr, int* status = nullptr);

// Split-K tall-skinny FP32 GEMM (skinny.cu): P[s](m, n) = sum_{k in split s}
// A[m*lda + k] X[n*ldx + k]; *S in: requested splits, out: planes written.
int skinny_splits(int M, int N, int K);
as_status launch_skinny_partial(cudaStream_t s, int M, int N, int K, int* S, const float* A, long long lda,
                                const float* X, long long ldx, float* P, long long ldp, long long plane);
// out[r*ldo + c] = sum_s P[s*plane + r*ldp + c], summed in FP64.
as_status launch_plane_sum(cudaStream_t s, const float* P, int S, long long plane, int rows, int cols, long long ldp,
                           float* out, long long ldo);
// G[p][r+t] = sum_s P[s][t*ldp + p] (FP64), mirrored to G[r+t][p] for p < r.
as_status launch_gram_reduce(cudaStream_t s, const float* P, long long ldp, long long plane, int S, int mrows, int r,
                             int b, double* G, int n2);
// G gains the Gram rows/columns of block rows [r, r+b) (FP64 combine of the splits).
as_status launch_gram_rows_skinny(cudaStream_t s, const float* C, int ldc, int d, int r, int b, double* G, int n2,
                                  float* P, size_t p_cap);

// Dump (the snapshot and residual step of Algorithm 4) for the first xi columns of W U / G W U
// (row-major n2 x k): Z = C'^T (WU)_xi, Y = (GWU)_xi^T C', C -= (GWU)_xi Z^T,
// G -= (GWU)_xi (GWU)_xi^T.  work: dump_work_doubles(d, n2, xi).
size_t dump_work_doubles(int d, int n2, int xi);
// Copies of C and G the dump keeps in step in the same passes (null: none):
// the BF16 levels of C (ld ldc), the FP32 mirror of G (ld n2) and its BF16
// levels (ld ldg, glevel elements apart).
struct DumpMirrors {
  __nv_bfloat16 *c0 = nullptr, *c1 = nullptr, *c2 = nullptr;
  float* gf = nullptr;
  __nv_bfloat16* gb = nullptr;
  long long glevel = 0;
  int ldg = 0;
};
as_status launch_dump(cudaStream_t s, float* C, int ldc, int d, int r, double* G, int n2, const double* WU,
                      const double* GWU, int k, int xi, float* Z, float* Y, double* work, const DumpMirrors& mir);

// FP32 mirror of the leading m x m block of G for the rows/columns at or past
// `valid` (the leading valid x valid block is already mirrored).
as_status launch_gf_mirror(cudaStream_t s, const double* G, float* Gf, int n2, int valid, int m);

// tcgen05 GEMM operand (umma.cu): TMA tensor maps over the BF16 levels of a
// split FP32 matrix (m[0] = hi; m[1], m[2] the lower levels), K innermost,
// box 64 x box_rows.
struct UmmaOperand {
  CUtensorMap m[3];
};

// Scratch of the GEMM paths (split-K planes, also used by the FP32 Gram rows).
struct BatchBuffers {
  float* P;       // p_cap floats
  int max_splits;
};

// Buffers of the persistent batched iterations (batch_persist.cu).
struct PersistBuffers {
  float* Y;       // 2 buffers of ybuf floats, columns of ldy floats
  long long ybuf;
  int ldy;
  size_t ycols;   // columns per buffer (batch_persist_ycols(bmax))
  int bmax;
  float* X;       // n2 x ycols, column-major (ld n2): final basis of every pair
  float* part;    // batch_persist_part_floats(bmax)
  unsigned* cnt;  // grid-barrier counter
  double* sig2;   // bmax   power-iteration estimates
  double* ritz;   // 2*bmax the two Ritz values of the k = 2 step
};
size_t batch_persist_ycols(int bmax);
size_t batch_persist_part_floats(int bmax);
// Column of the first vector of row t's simultaneous-iteration pair.
int batch_si_col(int nb, int t);

// Block-speculative power iteration (Algorithm 1) and first doubling step
// (k = 2) of the simultaneous iteration (Algorithm 2) for rows t = 0..nb-1 of
// a block whose row t sees the leading r0+t+1 rows of G; Gf is the FP32
// mirror of G's leading (r0+nb) x (r0+nb) block.  One cooperative launch;
// a grid-barrier wait that gives up sets AS_ETIMEOUT in *status.
as_status launch_batch_persist(cudaStream_t s, const float* Gf, int n2, int r0, int nb, int k_pi, int q, Key key,
                               uint64_t i0, const PersistBuffers& pb, int* status, Prof* prof = nullptr);

// One block of one sketch for a grouped launch of the FP32 persistent kernel.
struct BatchJob {
  const float* Gf;
  int n2, r0, nb, k_pi, q;
  Key key;
  uint64_t i0;
  PersistBuffers pb;
  int* status;
};
// CTAs a grouped launch may hold (one per SM), and a job's tiles (0: it
// cannot join a group).
int batch_group_capacity();
int batch_group_tiles(const BatchJob& j);
// The jobs' blocks in one cooperative launch on stream s (at most 32 jobs,
// their tiles within the capacity); cnt is the launch's barrier counter.
// Each job's results equal those of its own launch_batch_persist.
as_status launch_batch_group(cudaStream_t s, const BatchJob* jobs, int n, unsigned* cnt);

// x^(0) and Pi of every row of a block into buffer 1 of pb.Y (FP32), as the
// persistent kernels read them at iteration 0.
void launch_persist_fill(cudaStream_t s, const PersistBuffers& pb, int mmax, int nb, int npi, int r0, Key key,
                         uint64_t i0);

// Tensor-core form of the batched iterations (tensor precision forms):
// BF16 levels of G (mirrored like the FP32 copy), of the batch vectors, and
// the K-split partial products.
struct TcBatchBuffers {
  __nv_bfloat16* Gb;    // 3 levels of n2p x n2p (row-major, ld ldg), glevel elements apart
  long long glevel;
  int ldg;
  UmmaOperand mG;       // tensor maps of the G levels (box 64 x 128)
  __nv_bfloat16* Yb;    // 3 levels x 2 buffers x ycols columns of ldyb
  long long yblevel;
  int ldyb;
  float* part;
};
size_t batch_tc_part_floats(int n2, int ycols);
// BF16 levels of the new rows and columns of G, and with Gf also the FP32 mirror.
as_status launch_tc_mirror(cudaStream_t s, const double* G, int n2, int valid, int m, const TcBatchBuffers& tb,
                           float* Gf = nullptr);
// Runs the block on tcgen05 when its shape allows (kpad >= 256, at most 192
// columns, a co-resident grid); *used = false leaves it to launch_batch_persist.
// The starting vectors of a block's tcgen05 batch (and its flags cleared) on
// stream s, ahead of launch_batch_tc(..., prefilled = true); *done = false
// when the block's shape does not take the tcgen05 batch.
as_status launch_batch_tc_prefill(cudaStream_t s, int n2, int r0, int nb, Key key, uint64_t i0,
                                  const PersistBuffers& pb, const TcBatchBuffers& tb, bool* done);
as_status launch_batch_tc(cudaStream_t s, int n2, int r0, int nb, int k_pi, int q, Key key, uint64_t i0,
                          const PersistBuffers& pb, const TcBatchBuffers& tb, int npass, int* status, Prof* prof,
                          bool* used, bool prefilled = false);

// FP64 single-row power iteration and simultaneous iteration built from
// multi-block products (any buffer size).  x, y: n2 doubles; zero: 1 int.
as_status launch_power_iteration_f64(cudaStream_t s, const double* G, int n2, int m, int k_pi, Key key,
                                     uint64_t i, double* x, double* y, int* zero, double* sig2, uint64_t jsub = 0);
// R = G - (GWU)_xi (GWU)_xi^T on the leading m x m block (ld n2): the Gram of
// the residual C' - C' Z Z^T (probability amplification, Algorithm 7).
as_status launch_residual_gram(cudaStream_t s, const double* G, int n2, int m, const double* GWU, int k, int xi,
                               double* R);
as_status launch_simul_iter_f64(cudaStream_t s, const double* G, int n2, int m, int k, int q, Key key, uint64_t i,
                                int j, const SiBuffers& b, int* status);

// The Rayleigh-Ritz step of Algorithm 2 (k = 2) in FP64 on the iterated
// basis that the batched pass left in columns col0, col0+1 of X (FP32).
as_status launch_si_rr_from_batch(cudaStream_t s, const double* G, int n2, int m, const float* X, int col0,
                                  const SiBuffers& b, int* status);

bool umma_available();
as_status umma_make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int kdim, long long ld, int box_rows);
int umma_bn_for(int N);
// out[z*plane + m*som + n*son] = sum_{k in split z} A(m,k) B(b_row0 + n, k); npass 1 (BF16),
// 3 (two-level split-BF16) or 6 (three-level split-BF16, FP32-equivalent operands).
// precise = true (bn must be 64): one accumulator per K = 16 step of a stage
// (for products that write sketch state; use 64-element K splits).
as_status launch_umma_gemm(cudaStream_t s, const UmmaOperand& A, const UmmaOperand& B, int M, int N, int K, int bn,
                           int npass, int splits, int b_row0, float* out, long long som, long long son, long long plane,
                           int* err, bool precise = false);
// BF16 levels of an FP32 matrix (hi, lo, and optionally a third level lo2),
// optionally transposed (dst(c, r) = src(r, c)).
as_status launch_split_bf16(cudaStream_t s, const float* src, long long lds, int rows, int cols, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, long long ldd, bool transpose, __nv_bfloat16* lo2 = nullptr);

// Low-rank route of the query (lowrank.cu): out = Z^T (Z: d x xi row-major);
// W' = D W D and H' = D^-1 H D^-1 from W = F F^T (kind[i] = {0: a row of C,
// 1: a row of Z_j^T, 2: a row of Y_j; first row of Z_j^T; xi_j}); the core
// K = L^1/2 sym(T) L^1/2 from T = U_r^T H' U_r; column scaling by lam^-1/2,
// row scaling by D; the l largest eigenvalues of B from those of K.
as_status launch_transpose_f32(cudaStream_t s, const float* Z, int d, int xi, float* out, long long ldo);
as_status launch_f32_to_f64(cudaStream_t s, const float* in, size_t n, double* out);
as_status launch_lr_scale(cudaStream_t s, const double* W, int n, const int4* kind, double* Ws, double* Hs);
as_status launch_lr_core(cudaStream_t s, const double* T, int ldt, const double* lam, int r, double* K);
as_status launch_lr_colscale(cudaStream_t s, double* U, int n, int ldu, const double* lam, int r);
as_status launch_lr_rowscale(cudaStream_t s, const double* W, int n, double* P, int m);
as_status launch_lr_lambda(cudaStream_t s, const double* mu, int lp, int ell, double* lam_out);

// Launch-shape autotuner (tune.cu): the fastest of `choices` for (device,
// kernel, key), timed on the first call's inputs by running run(choice); the
// choice is cached per key.  *ran = true when run(result) already produced
// this call's outputs.  AS_TUNE=0 in the environment returns choices[0].
int tune_pick(cudaStream_t s, const char* kernel, long long key, const int* choices, int n,
              const std::function<as_status(int)>& run, as_status* st, bool* ran);

// Library-internal access to a sketch for the runtimes built on sketches
// (engine.cu): stream, rows fed, the snapshot queue's times (the sketch's own
// row indices), the windowed query Gram, raw-row Grams, dropping the oldest
// snapshots, and the eigen-shrink of a device B (the eigen-shrink of Algorithm 5).
// Runs f(0) .. f(n-1) on the library's worker threads and waits for all.
void run_parallel(int n, const std::function<void(int)>& f);
// Several sketches updated together through the device's launch combiner
// (engine.cu): combined_begin returns the device's combiner as a token; each
// sketch's host thread brackets its updates with combined_enter/leave and
// calls sk_update_combined (sketch_update whose FP32 batched iterations share
// grouped launches with the other sketches' ready blocks).
as_status combined_begin(int dev, void** token);
void combined_enter(void* token);
void combined_leave(void* token);
as_status sk_update_combined(as_sketch* h, const float* rows, int64_t n, int64_t ld, void* token);
cudaStream_t sk_stream(const as_sketch* h);
int sk_device(const as_sketch* h);
int64_t sk_device_bytes(const as_sketch* h);
int64_t sk_rows(const as_sketch* h);
int sk_snap_count(const as_sketch* h);
int64_t sk_snap_t(const as_sketch* h, int k);
as_status sk_window_gram(as_sketch* h, int64_t lb, double* B);
as_status sk_add_rows_gram(as_sketch* h, const float* R, int k, int64_t ld, double* B);
as_status sk_drop_front(as_sketch* h, int count);
as_status sk_eig_shrink(as_sketch* h, double* B, float* out, int64_t ldo);
// FP64 squared norms of n rows (host or device, row stride ld) into out.
as_status row_norms_f64(const float* rows, long long n, long long ld, int d, cudaStream_t s, double* out);

// Query helpers.
as_status launch_shrink_rows(cudaStream_t s, int d, int ell, const double* lam, const double* V, int ldv,
                             float* out, long long ldo);

}  // namespace as
