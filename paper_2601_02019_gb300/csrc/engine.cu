// The sketch state machine and the C ABI (include/aerosketch.h).
//
// Device state of one sketch:
//   C      2l x ldc FP32  residual buffer (rows >= r are zero)
//   G      2l x 2l  FP64  Gram C C^T of the stored buffer
//   arena  FP32           snapshot store: for each snapshot Z (d x xi, row-major)
//                         followed by Y = Z^T C'^T C' (xi x d, row-major)
// The host walks Algorithm 4 block by block; every arithmetic step runs in the
// kernels, and the host reads back only the scalars that decide the branches
// (||a_i||^2, the power-iteration estimates, the Ritz values).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <new>
#include <unordered_map>
#include <vector>

#include "eig.cuh"
#include "kernels.cuh"

using namespace as;

namespace {

struct Snap {
  size_t off;  // offset in floats of Z in the arena; Y follows at off + d*xi
  int xi;
  int64_t s, t;
};

// as_inject_alloc_failure: allocations left before the one that fails (-1: off).
std::atomic<int64_t> g_fail_after{-1};

template <typename T>
as_status dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (g_fail_after.load(std::memory_order_relaxed) >= 0 && g_fail_after.fetch_sub(1) == 0) return AS_ENOMEM;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) { cudaGetLastError(); *p = nullptr; return AS_ENOMEM; }
  return AS_OK;
}

int ceil_log2(int64_t x) {  // smallest c with 2^c >= x, x >= 1
  int c = 0;
  while ((int64_t(1) << c) < x) ++c;
  return c;
}

}  // namespace

namespace as {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace as

namespace {

const char* const kProfNames[PK_COUNT] = {"batch_persist",     "batch_prep",        "eig_fp64",
                                          "fd_rebuild_gemm",   "gram_rows_gemm",    "ingest",
                                          "event_row_fp64",    "eig_tridiag",       "eig_bisect_invit",
                                          "eig_backtransform", "batch_tc"};

// CUDA-event timer per kernel class; pairs are resolved lazily.
struct EventProf final : Prof {
  struct Pending { int cls; cudaEvent_t a, b; double flops, bytes, issued; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[PK_COUNT] = {};
  double ms[PK_COUNT] = {}, flops[PK_COUNT] = {}, bytes[PK_COUNT] = {}, issued[PK_COUNT] = {};
  cudaEvent_t open_ev[PK_COUNT] = {};
  uint32_t mask = ~0u;   // classes bracketed with events (sketch_profile_select)

  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int cls, cudaStream_t s) override {
    if (!((mask >> cls) & 1u)) return;
    open_ev[cls] = get();
    cudaEventRecord(open_ev[cls], s);
  }
  void end(int cls, cudaStream_t s, double f, double b, double iss = -1.0) override {
    if (!((mask >> cls) & 1u)) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, s);
    pending.push_back(Pending{cls, open_ev[cls], e, f, b, iss < 0.0 ? f : iss});
    if (pending.size() > 8192) resolve();
  }
  void add_work(int cls, double f) override { flops[cls] += f; }
  void resolve() {
    for (Pending& p : pending) {
      cudaEventSynchronize(p.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, p.a, p.b);
      ms[p.cls] += t;
      launches[p.cls] += 1;
      flops[p.cls] += p.flops;
      bytes[p.cls] += p.bytes;
      issued[p.cls] += p.issued;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    resolve();
    for (int c = 0; c < PK_COUNT; ++c) { launches[c] = 0; ms[c] = flops[c] = bytes[c] = issued[c] = 0; }
  }
  ~EventProf() override {
    for (Pending& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

// Buffer sizes (2l) from which the FP64 single-row iterations spread over
// many blocks, and from which the FD shrink uses the GPU-wide df64
// eigensolver; below them one block does the work in FP64.  FP64 runs at a
// small fraction of the FP32 rate on this part, so one block is the slower
// choice at every size measured (2l = 32 .. 256: 1.2x to 3x per sketch), and
// both thresholds default to 0; the one-block forms stay for the build-time
// choice and for as_symeig.
#ifndef AS_MULTI_ROW_MIN
#define AS_MULTI_ROW_MIN 0
#endif
#ifndef AS_EIG_LARGE_MIN
#define AS_EIG_LARGE_MIN 0
#endif
constexpr int kMultiRowMin = AS_MULTI_ROW_MIN;
constexpr int kEigLargeMin = AS_EIG_LARGE_MIN;

struct as_sketch {
  as_config cfg{};
  int d = 0, ell = 0, n2 = 0, ldc = 0, k_pi = 0, q = 0, jmax = 0, mode = 0;
  int amp_r = 0, amp_s = 0, q_amp = 0;   // probability amplification (Algorithm 7); amp_r = 0: off
  int dev = 0;                           // the CUDA device the state lives on
  double eps = 0, eps_si = 0, theta = 0;
  cudaStream_t s = nullptr;
  Key key{};
  // device buffers
  float *C = nullptr, *Cnew = nullptr, *Wfd = nullptr, *stage = nullptr, *Gf = nullptr;
  double *G = nullptr, *Gtmp = nullptr, *lam = nullptr, *U = nullptr, *eigw = nullptr, *scal = nullptr;
  double *x64 = nullptr, *y64 = nullptr, *norm2 = nullptr, *dwork = nullptr;
  size_t dwork_cap = 0;
  size_t p_cap = 0;
  int *bad = nullptr, *dstatus = nullptr, *zero = nullptr;
  SiBuffers si{};
  BatchBuffers bb{};
  int bmax = 64, bnext = 64;
  bool big = false;      // multi-block FP64 single-row iterations (2l >= kMultiRowMin)
  bool big_eig = false;  // the GPU-wide df64 eigensolver for the FD shrink (2l >= kEigLargeMin)
  double* h_buf = nullptr;  // pinned host scratch for branch scalars
  int stage_rows = 0;
  // host mirror of the control state
  int r = 0;
  int64_t T = 0;
  double F = 0.0;
  float* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  std::vector<Snap> snaps;
  // absorbed terms (d x d FP64): snapshots sent here by sketch_send_snapshots
  // and sketches merged in by sketch_merge; allocated on first use
  double* Bx = nullptr;
  double *sx_yz = nullptr, *sx_t = nullptr;   // scratch of the snapshot-term products
  int sx_cap = 0;                              // xi capacity of the scratch
  as_stats st{};
  std::vector<as_event> trace;
  size_t dev_bytes = 0;
  std::mutex mu;
  EventProf* prof = nullptr;  // AS_PROFILE
  // tensor-core forms (AS_BF16, AS_BF16X3)
  bool tc = false;
  int dpass = 1;            // passes of the d-side products (1 BF16, 3 split-BF16)
  int n2p = 0;              // n2 rounded up to 64
  int rows_pad = 0;         // row counts of the BF16 buffers, >= 256
  __nv_bfloat16 *Chi = nullptr, *Clo = nullptr, *Cthi = nullptr, *Ctlo = nullptr, *Wh = nullptr, *Wl = nullptr;
  __nv_bfloat16 *Cl2 = nullptr, *Ctl2 = nullptr, *Wl2 = nullptr;   // third BF16 level (AS_BF16X6)
  float* Prb = nullptr;     // split-K planes of the FD rebuild (tensor forms)
  size_t prb_cap = 0;
  UmmaOperand mCA{}, mCB64{}, mCB256{}, mWA{}, mCtB{};
  // persistent batched iterations
  PersistBuffers pb{};
  bool tcb = false;         // tcgen05 form of the batched iterations (tensor forms, 2l >= 256)
  TcBatchBuffers tb{};
  int gf_valid = 0;         // leading rows/columns of Gf that equal G (FP32-rounded)
  cudaEvent_t comb_ev = nullptr;   // a deferred block's launch phase is done (launch combiner)
  // side stream for the starting vectors of a block's tcgen05 batch, filled
  // while the block's rows are ingested and its Gram rows formed
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_blk = nullptr, ev_fill = nullptr;
};

namespace {

void free_all(as_sketch* h) {
  float* fp[] = {h->C, h->Cnew, h->Wfd, h->stage, h->arena, h->Gf, h->bb.P, h->Prb, h->pb.Y, h->pb.X, h->pb.part};
  for (float* p : fp) if (p) cudaFree(p);
  double* dp[] = {h->G, h->Gtmp, h->lam, h->U, h->eigw, h->scal, h->si.Y, h->si.GY, h->si.S, h->si.V,
                  h->si.eigw, h->si.ritz, h->si.WU, h->si.GWU, h->si.tmp, h->x64, h->y64, h->norm2, h->dwork,
                  h->pb.sig2, h->pb.ritz};
  for (double* p : dp) if (p) cudaFree(p);
  if (h->bad) cudaFree(h->bad);
  if (h->dstatus) cudaFree(h->dstatus);
  if (h->zero) cudaFree(h->zero);
  if (h->pb.cnt) cudaFree(h->pb.cnt);
  double* xp[] = {h->Bx, h->sx_yz, h->sx_t};
  for (double* p : xp) if (p) cudaFree(p);
  __nv_bfloat16* bp[] = {h->Chi, h->Clo, h->Cthi, h->Ctlo, h->Wh, h->Wl, h->Cl2, h->Ctl2, h->Wl2, h->tb.Gb, h->tb.Yb};
  for (__nv_bfloat16* p : bp) if (p) cudaFree(p);
  if (h->tb.part) cudaFree(h->tb.part);
  if (h->h_buf) cudaFreeHost(h->h_buf);
  if (h->comb_ev) cudaEventDestroy(h->comb_ev);
  if (h->ev_blk) cudaEventDestroy(h->ev_blk);
  if (h->ev_fill) cudaEventDestroy(h->ev_fill);
  if (h->s2) cudaStreamDestroy(h->s2);
  delete h->prof;
  h->prof = nullptr;
}

as_status sync_status(as_sketch* h) {
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  int ds = 0;
  AS_CUDA_TRY(cudaMemcpy(&ds, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
  return (as_status)ds;
}

// Read `n` doubles from device memory into the pinned host buffer (synchronising).
as_status fetch(as_sketch* h, const double* src, int n) {
  AS_CUDA_TRY(cudaMemcpyAsync(h->h_buf, src, n * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  return AS_OK;
}

// Room for `extra` more floats in the snapshot store: the capacity doubles
// (from 8 d l floats), or with exact = true grows to exactly what is needed.
as_status arena_reserve(as_sketch* h, size_t extra, bool exact = false) {
  if (h->arena_used + extra <= h->arena_cap) return AS_OK;
  size_t cap = h->arena_cap ? h->arena_cap : (size_t)8 * h->d * h->ell;
  while (cap < h->arena_used + extra) cap *= 2;
  if (exact) cap = h->arena_used + extra;
  float* na = nullptr;
  as_status st = dalloc(&na, cap);
  if (st != AS_OK) return st;
  if (h->arena_used)
    AS_CUDA_TRY(cudaMemcpyAsync(na, h->arena, h->arena_used * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  if (h->arena) cudaFree(h->arena);
  h->dev_bytes += (cap - h->arena_cap) * sizeof(float);
  h->arena = na;
  h->arena_cap = cap;
  return AS_OK;
}

// BF16 (hi, lo) shadows of C rows [r0, r1) for the tensor-core forms.
as_status tc_split_rows(as_sketch* h, int r0, int r1) {
  if (!h->tc || r1 <= r0) return AS_OK;
  return launch_split_bf16(h->s, h->C + (size_t)r0 * h->ldc, h->ldc, r1 - r0, h->ldc, h->Chi + (size_t)r0 * h->ldc,
                           h->Clo + (size_t)r0 * h->ldc, h->ldc, false,
                           h->Cl2 ? h->Cl2 + (size_t)r0 * h->ldc : nullptr);
}

// Longest K range of one split of the products that write state (Gram rows,
// FD rebuild): longer ranges are split and the partial planes summed in FP64.
// In the precise mode of the tcgen05 GEMM each of the four K = 16 MMAs of a
// 64-wide tile has its own accumulator, so a 256-element split costs each
// accumulator three truncating accumulate steps; this keeps the accumulation
// error near that of the FP32 form (FP32 partial sums of 64, combined in FP64)
// while writing a quarter of the planes of 64-element splits.
constexpr int kTcStateChunk = 256;

as_status ensure_prb(as_sketch* h, size_t need) {
  if (need <= h->prb_cap) return AS_OK;
  if (h->Prb) cudaFree(h->Prb);
  h->Prb = nullptr;
  h->dev_bytes -= h->prb_cap * sizeof(float);
  h->prb_cap = 0;
  as_status st = dalloc(&h->Prb, need);
  if (st == AS_OK) {
    h->dev_bytes += (need - h->prb_cap) * sizeof(float);
    h->prb_cap = need;
  }
  return st;
}

// G gains the Gram rows/columns of rows [r, r+b) through the tcgen05 GEMM
// (A = C rows [0, r+b), B = C rows [r, r+b), K = d) and the split reduction.
as_status tc_gram_rows(as_sketch* h, int r, int b, const UmmaOperand& Bmap, int bn) {
  const int M = r + b;
  const int mt = (M + 127) / 128, nt = (b + bn - 1) / bn, ktiles = h->ldc / 64;
  int S = std::max(1, std::min((2 * 152 + mt * nt - 1) / (mt * nt), ktiles));
  S = std::max(S, (h->ldc + kTcStateChunk - 1) / kTcStateChunk);
  const int klen = ((ktiles + S - 1) / S) * 64;
  S = (h->ldc + klen - 1) / klen;
  as_status st = AS_OK;
  float* P = h->bb.P;
  const size_t need = (size_t)S * b * M;
  if (need > h->p_cap) {
    st = ensure_prb(h, need);
    if (st != AS_OK) return st;
    P = h->Prb;
  }
  st = launch_umma_gemm(h->s, h->mCA, Bmap, M, b, h->ldc, bn, h->dpass, S, r, P, 1, M, (long long)b * M, h->dstatus,
                        bn == 64);
  if (st != AS_OK) return st;
  return launch_gram_reduce(h->s, P, M, (long long)b * M, S, M, r, b, h->G, h->n2);
}

// The FD shrink of Algorithm 4 (Section 2.3) on the full buffer, through its Gram.
as_status fd_shrink(as_sketch* h) {
  const int n2 = h->n2, ell = h->ell, d = h->d;
  AS_CUDA_TRY(cudaMemcpyAsync(h->Gtmp, h->G, (size_t)n2 * n2 * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
  if (h->prof) h->prof->begin(PK_EIG, h->s);
  as_status st = h->big_eig ? launch_eig_large(h->s, n2, h->Gtmp, n2, ell, h->lam, h->U, ell, h->eigw, h->prof, h->dstatus)
                         : launch_eig(h->s, n2, h->Gtmp, n2, ell, h->lam, h->U, ell, h->eigw);
  if (st != AS_OK) return st;
  // tridiagonalisation 4/3 n^3 + back-transformation 2 n^2 nev; G read once
  if (h->prof)
    h->prof->end(PK_EIG, h->s, 4.0 / 3.0 * (double)n2 * n2 * n2 + 2.0 * (double)n2 * n2 * ell,
                 8.0 * (double)n2 * n2);
  if (h->prof) h->prof->begin(PK_REBUILD, h->s);
  st = launch_shrink_weights(h->s, n2, ell, h->lam, h->U, h->Wfd);
  if (st != AS_OK) return st;
  AS_CUDA_TRY(cudaMemsetAsync(h->Cnew, 0, (size_t)n2 * h->ldc * sizeof(float), h->s));
  if (ell > 1 && h->tc) {
    // C' = W C~ on tcgen05: A = W (rows j, K = p), B = C~^T (rows c, K = p)
    st = launch_split_bf16(h->s, h->Wfd, n2, ell - 1, n2, h->Wh, h->Wl, h->n2p, false, h->Wl2);
    if (st == AS_OK) st = launch_split_bf16(h->s, h->C, h->ldc, n2, d, h->Cthi, h->Ctlo, h->n2p, true, h->Ctl2);
    // split K (the 2l buffer rows) into chunks of kTcStateChunk; planes summed in FP64
    int S = (h->n2p + kTcStateChunk - 1) / kTcStateChunk;
    const int klen = ((h->n2p / 64 + S - 1) / S) * 64;
    S = (h->n2p + klen - 1) / klen;
    const size_t need = (size_t)S * (ell - 1) * d;
    if (st == AS_OK) st = ensure_prb(h, need);
    if (st == AS_OK)
      st = launch_umma_gemm(h->s, h->mWA, h->mCtB, ell - 1, d, h->n2p, 64, h->dpass, S, 0, h->Prb, d, 1,
                            (long long)(ell - 1) * d, h->dstatus, true);
    if (st == AS_OK) st = launch_plane_sum(h->s, h->Prb, S, (long long)(ell - 1) * d, ell - 1, d, d, h->Cnew, h->ldc);
    if (st != AS_OK) return st;
  } else if (ell > 1) {
    st = gemm_strided<float, float, float>(h->s, ell - 1, d, n2, h->Wfd, n2, 1, h->C, h->ldc, 1, h->Cnew, h->ldc,
                                           1, 1.0, 0.0);
    if (st != AS_OK) return st;
  }
  std::swap(h->C, h->Cnew);
  AS_CUDA_TRY(cudaMemsetAsync(h->G, 0, (size_t)n2 * n2 * sizeof(double), h->s));
  if (ell > 1 && h->tc) {
    st = tc_split_rows(h, 0, n2);
    if (st == AS_OK) st = tc_gram_rows(h, 0, ell - 1, h->mCB64, 64);
    if (st != AS_OK) return st;
  } else if (ell > 1) {
    st = gemm_strided<float, float, double>(h->s, ell - 1, ell - 1, d, h->C, h->ldc, 1, h->C, 1, h->ldc, h->G, n2,
                                            1, 1.0, 0.0);
    if (st != AS_OK) return st;
  } else if (h->tc) {
    st = tc_split_rows(h, 0, n2);
    if (st != AS_OK) return st;
  }
  // C' = W C~ ((l-1) x 2l x d) and G = C' C'^T ((l-1)^2 x d); C~ read, C' written and read
  if (h->prof)
    h->prof->end(PK_REBUILD, h->s, 2.0 * (ell - 1) * (double)n2 * d + 2.0 * (ell - 1) * (double)(ell - 1) * d,
                 4.0 * ((double)n2 * d + 2.0 * (ell - 1) * (double)d));
  h->r = ell - 1;
  h->gf_valid = 0;
  h->st.shrinks++;
  return AS_OK;
}

as_status ensure_dwork(as_sketch* h, size_t need) {
  if (need <= h->dwork_cap) return AS_OK;
  if (h->dwork) cudaFree(h->dwork);
  h->dwork = nullptr;
  h->dev_bytes -= h->dwork_cap * sizeof(double);
  h->dwork_cap = 0;
  as_status st = dalloc(&h->dwork, need);
  if (st != AS_OK) return st;
  h->dev_bytes += need * sizeof(double);
  h->dwork_cap = need;
  return AS_OK;
}

// Largest sizes of the buffers that grow on demand: the dump work (xi <= l)
// and, for the tensor-core forms, the split-K planes of the Gram rows (at most
// ldc/64 planes of bmax x 2l) and of the FD rebuild (n2p/64 planes of (l-1) x d).
size_t dwork_max(const as_sketch* h) { return dump_work_doubles(h->d, h->n2, h->ell); }
size_t prb_max(const as_sketch* h) {
  if (!h->tc) return 0;
  return std::max((size_t)(h->ldc / 64) * h->bmax * h->n2, (size_t)(h->n2p / 64) * (h->ell - 1) * h->d);
}

// The snapshot and residual step of Algorithm 4 for the first xi columns of
// the last SI (k columns).
as_status dump(as_sketch* h, int xi, int k, int64_t i) {
  const int d = h->d, r = h->r, ldc = h->ldc, n2 = h->n2;
  as_status st = arena_reserve(h, (size_t)2 * d * xi);
  if (st != AS_OK) return st;
  float* Z = h->arena + h->arena_used;
  float* Y = Z + (size_t)d * xi;
  st = ensure_dwork(h, dump_work_doubles(d, n2, xi));
  if (st != AS_OK) return st;
  // the residual and the Gram downdate also refresh the BF16 levels of C and
  // the mirrors of G (FP32, and BF16 for the tcgen05 batch) in their passes
  DumpMirrors mir;
  if (h->tc) {
    mir.c0 = h->Chi;
    mir.c1 = h->Clo;
    mir.c2 = h->Cl2;
  }
  mir.gf = h->Gf;
  if (h->tcb) {
    mir.gb = h->tb.Gb;
    mir.glevel = h->tb.glevel;
    mir.ldg = h->tb.ldg;
  }
  st = launch_dump(h->s, h->C, ldc, d, r, h->G, n2, h->si.WU, h->si.GWU, k, xi, Z, Y, h->dwork, mir);
  if (st != AS_OK) return st;
  h->gf_valid = r;   // rows and columns [0, r) of both mirrors were rewritten with G
  const int64_t s_prev = h->snaps.empty() ? 1 : h->snaps.back().t + 1;
  h->snaps.push_back(Snap{h->arena_used, xi, s_prev, i});
  h->arena_used += (size_t)2 * d * xi;
  h->st.dumps++;
  h->st.snapshot_rank += xi;
  return AS_OK;
}

// FP64 power iteration (Algorithm 1) on the current state (first r rows).
as_status pi_f64(as_sketch* h, int64_t i, double* sig2) {
  as_status st = h->big ? launch_power_iteration_f64(h->s, h->G, h->n2, h->r, h->k_pi, h->key, (uint64_t)i, h->x64,
                                                     h->y64, h->zero, h->scal)
                        : launch_power_iteration(h->s, h->G, h->n2, h->r, h->k_pi, h->key, (uint64_t)i, h->scal);
  if (st != AS_OK) return st;
  st = fetch(h, h->scal, 1);
  if (st != AS_OK) return st;
  *sig2 = h->h_buf[0];
  return AS_OK;
}

// Algorithm 2 (FP64) for row i with k columns, q products and the test matrix
// at Philox sub-index jsub; the Ritz values land in h->h_buf[0..k).
as_status si_f64(as_sketch* h, int64_t i, int jsub, int k, int q) {
  as_status st = h->big ? launch_simul_iter_f64(h->s, h->G, h->n2, h->r, k, q, h->key, (uint64_t)i, jsub, h->si, h->dstatus)
                        : launch_simul_iter(h->s, h->G, h->n2, h->r, k, q, h->key, (uint64_t)i, jsub, h->si, h->dstatus);
  if (st != AS_OK) return st;
  h->st.si_runs++;
  return fetch(h, h->si.ritz, k);
}

// Algorithm 7 in place of Algorithm 4's simultaneous iteration (doubling step
// j, k columns):
// amp_r simultaneous iterations with eps_SI = 0.2, SI h drawing its test matrix
// at sub-index j + 64 (h-1); each is scored by the largest of amp_s power-
// iteration estimates (start vectors at sub-index 64 h + g) of the top
// eigenvalue of its residual C' - C' Z_h Z_h^T, whose Gram G - (G WU)(G WU)^T
// is formed in Gtmp (Z_h restricted to its xi_h columns at or above theta).
// The first minimum is kept; its WU, GWU and Ritz values are left in h->si and
// h->h_buf.  *chosen = the kept h.
as_status amplified_si(as_sketch* h, int64_t i, int j, int k, double theta, int* chosen) {
  double best = 0.0;
  int hbest = 0;
  for (int hh = 1; hh <= h->amp_r; ++hh) {
    as_status st = si_f64(h, i, j + 64 * (hh - 1), k, h->q_amp);
    if (st != AS_OK) return st;
    int xi = 0;
    for (int c = 0; c < k; ++c)
      if (h->h_buf[c] >= theta && h->h_buf[c] > 0.0) ++xi;
    st = launch_residual_gram(h->s, h->G, h->n2, h->r, h->si.GWU, k, xi, h->Gtmp);
    for (int g = 1; g <= h->amp_s && st == AS_OK; ++g) {
      const uint64_t jsub = 64 * (uint64_t)hh + (uint64_t)g;
      st = h->big ? launch_power_iteration_f64(h->s, h->Gtmp, h->n2, h->r, h->k_pi, h->key, (uint64_t)i, h->x64,
                                               h->y64, h->zero, h->scal + (g - 1), jsub)
                  : launch_power_iteration(h->s, h->Gtmp, h->n2, h->r, h->k_pi, h->key, (uint64_t)i,
                                           h->scal + (g - 1), jsub);
    }
    if (st == AS_OK) st = fetch(h, h->scal, h->amp_s);
    if (st != AS_OK) return st;
    double ch = 0.0;
    for (int g = 0; g < h->amp_s; ++g) ch = std::max(ch, h->h_buf[g]);
    if (hbest == 0 || ch < best) {
      best = ch;
      hbest = hh;
    }
  }
  *chosen = hbest;
  // the last SI's buffers are the kept ones unless an earlier h won
  if (hbest == h->amp_r) return fetch(h, h->si.ritz, k);
  return si_f64(h, i, j + 64 * (hbest - 1), k, h->q_amp);
}

// The decision part of Algorithm 4 for row i on the current state (the
// power-iteration gate, the doubling simultaneous iteration, the selection of
// xi components and the dump), in FP64; Algorithm 7 replaces each
// simultaneous iteration when amplification is on.  The batched pass has
// usually decided the gate already: outside its tie band the outcome comes in
// as known_gate (with its estimate sig2) and no FP64 power iteration runs.
// For the first doubling step (k = 2) of a large buffer the batch also hands
// over its iterated basis (column batch_col of the batch's X), and only the
// FP64 Rayleigh-Ritz step is redone.  A dump ends the doubling loop as soon
// as the k-th Ritz value falls below theta; xi = 0 leaves the state as it is.
as_status finish_row(as_sketch* h, int64_t i, double theta, int known_gate, double sig2, int batch_col = -1,
                     int batch_ld = 0) {
  as_status st = AS_OK;
  if (known_gate < 0) {
    st = pi_f64(h, i, &sig2);
    if (st != AS_OK) return st;
  }
  const bool gate = (known_gate >= 0) ? (known_gate == 1) : (sig2 >= theta / 2.0 && sig2 > 0.0);
  if (!gate) return AS_OK;
  h->st.gates++;
  as_event ev{};
  ev.i = i;
  ev.sig2_pi = sig2;
  ev.theta = theta;
  for (int j = 1; j <= h->jmax; ++j) {
    const int k = std::min(std::min(1 << std::min(j, 30), h->ell), h->d);   // k = 2, 4, ... capped at min(l, d)
    if (h->amp_r > 0) {
      int hk = 0;
      st = amplified_si(h, i, j, k, theta, &hk);
      if (st == AS_OK && j <= 16) ev.amp_choice |= (uint64_t)hk << (4 * (j - 1));
    } else if (j == 1 && k == 2 && batch_col >= 0) {
      st = launch_si_rr_from_batch(h->s, h->G, h->n2, h->r, h->pb.X, batch_col, h->si, h->dstatus);
      if (st == AS_OK) st = fetch(h, h->si.ritz, k);
      h->st.si_runs++;
    } else {
      st = si_f64(h, i, j, k, h->q);
    }
    if (st != AS_OK) return st;
    const double* ritz = h->h_buf;   // Ritz values, descending
    ev.ritz_1 = ritz[0];
    ev.ritz_k = ritz[k - 1];
    if (ritz[k - 1] < theta) {   // the subspace holds every component at or above theta
      int xi = 0;
      for (int c = 0; c < k; ++c)
        if (ritz[c] >= theta && ritz[c] > 0.0) ++xi;
      ev.j_stop = j;
      ev.xi = xi;
      if (xi >= 1) {
        st = dump(h, xi, k, i);
        if (st != AS_OK) return st;
      }
      break;
    }
  }
  if (h->cfg.flags & AS_TRACE_DECISIONS) h->trace.push_back(ev);
  return AS_OK;
}

// One block of Algorithm 8 + Algorithm 4 over rows src[0..navail) (device,
// row stride d).  Rows are appended speculatively; the batched FP32 pass finds
// the first row whose decision changes the state (a dump, or the row that
// fills the buffer); rows before it are committed, the state is cut back to
// that row, and it is finished in FP64.  Returns the rows consumed in *used.
constexpr double kTieBand = 1e-4;

// A block between its launch phase and its decision phase.
struct BlockCtx {
  int b = 0, nbb = 0, r0 = 0;
  bool deferred = false;   // the FP32 batched iterations are left to the caller (a grouped launch)
  int batch_cls = -1;      // profiler class of the block's own batched launch (-1: none or grouped)
};

// Launch phase of one block (Algorithm 8's threshold update and Algorithm 4's
// insert, gate and first doubling step for every row, speculatively): ingest,
// Gram rows, mirrors of G and the batched iterations.  With defer, a block
// that would run the FP32 persistent kernel is left for a grouped launch
// (block_job describes it).
as_status block_prepare(as_sketch* h, const float* src, int64_t navail, BlockCtx& c, bool defer) {
  const int d = h->d, n2 = h->n2, r0 = h->r;
  const int b = (int)std::min<int64_t>({navail, (int64_t)(n2 - r0), (int64_t)h->bnext});
  c.b = b;
  c.r0 = r0;
  c.deferred = false;
  // tensor forms: the batch's starting vectors on the side stream, after all
  // work already on the sketch's stream, overlapping ingest and Gram rows
  const int nbb_early = (r0 + b == n2) ? b - 1 : b;
  bool prefilled = false;
  if (h->tcb && nbb_early > 0) {
    if (!h->s2) {
      AS_CUDA_TRY(cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking));
      AS_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_blk, cudaEventDisableTiming));
      AS_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fill, cudaEventDisableTiming));
    }
    AS_CUDA_TRY(cudaEventRecord(h->ev_blk, h->s));
    AS_CUDA_TRY(cudaStreamWaitEvent(h->s2, h->ev_blk, 0));
    as_status pst = launch_batch_tc_prefill(h->s2, n2, r0, nbb_early, h->key, (uint64_t)(h->T + 1), h->pb, h->tb,
                                            &prefilled);
    if (pst != AS_OK) return pst;
    AS_CUDA_TRY(cudaEventRecord(h->ev_fill, h->s2));
  }
  if (h->prof) h->prof->begin(PK_INGEST, h->s);
  as_status st = launch_ingest(h->s, src, d, b, d, h->C, h->ldc, r0, h->norm2, h->bad);
  if (st != AS_OK) return st;
  if (h->prof) h->prof->end(PK_INGEST, h->s, 2.0 * b * (double)d, 8.0 * b * (double)d);
  st = tc_split_rows(h, r0, r0 + b);
  if (st != AS_OK) return st;
  // the insert for the whole block: G gains the new rows and columns (a rejected
  // row was ingested as zeros, so nothing non-finite reaches the products)
  if (h->prof) h->prof->begin(PK_GRAM, h->s);
  st = h->tc ? tc_gram_rows(h, r0, b, h->mCB64, 64)
             : launch_gram_rows_skinny(h->s, h->C, h->ldc, d, r0, b, h->G, n2, h->bb.P, h->p_cap);
  if (st != AS_OK) return st;
  h->gf_valid = std::min(h->gf_valid, r0);
  if (h->prof)
    h->prof->end(PK_GRAM, h->s, 2.0 * (r0 + b) * (double)b * d, 4.0 * (r0 + b) * (double)d + 8.0 * (r0 + b) * b);
  const bool fills_all = (r0 + b == n2);
  const int nbb = fills_all ? b - 1 : b;   // batched rows (the filling row needs the shrink first)
  c.nbb = nbb;
  if (nbb > 0) {
    if (h->prof) h->prof->begin(PK_BATCH_ORTH, h->s);
    // both mirrors from one read of G when the tensor batch is on
    st = h->tcb ? launch_tc_mirror(h->s, h->G, n2, h->gf_valid, r0 + nbb, h->tb, h->Gf)
                : launch_gf_mirror(h->s, h->G, h->Gf, n2, h->gf_valid, r0 + nbb);
    if (st != AS_OK) return st;
    if (h->prof) {
      const double nm = (double)(r0 + nbb) * (r0 + nbb) - (double)h->gf_valid * h->gf_valid;
      h->prof->end(PK_BATCH_ORTH, h->s, 0.0, 12.0 * nm);
    }
    h->gf_valid = r0 + nbb;
    // tensor forms: the tcgen05 form of the batched iterations where the block's
    // shape allows it, else the FP32 persistent kernel.  Three split-BF16
    // passes (about 1e-5 relative) suffice in every form: the batch only
    // decides (gate and k = 2 stop tests, each re-decided in FP64 within a
    // 1e-4 relative tie band) and hands the event row a starting basis whose
    // Rayleigh-Ritz step is redone in FP64.
    bool on_tc = false;
    if (h->tcb && h->s2) AS_CUDA_TRY(cudaStreamWaitEvent(h->s, h->ev_fill, 0));   // the side stream's writes
    if (h->tcb) {
      st = launch_batch_tc(h->s, n2, r0, nbb, h->k_pi, h->q, h->key, (uint64_t)(h->T + 1), h->pb, h->tb,
                           3, h->dstatus, h->prof, &on_tc, prefilled);
      if (st != AS_OK) return st;
    }
    if (on_tc) c.batch_cls = PK_BATCH_TC;
    if (!on_tc) {
      if (defer) {
        c.deferred = true;
      } else {
        st = launch_batch_persist(h->s, h->Gf, n2, r0, nbb, h->k_pi, h->q, h->key, (uint64_t)(h->T + 1), h->pb,
                                  h->dstatus, h->prof);
        if (st != AS_OK) return st;
        c.batch_cls = PK_BATCH_GEMM;
      }
    }
  }
  return AS_OK;
}

BatchJob block_job(const as_sketch* h, const BlockCtx& c) {
  BatchJob j{};
  j.Gf = h->Gf;
  j.n2 = h->n2;
  j.r0 = c.r0;
  j.nb = c.nbb;
  j.k_pi = h->k_pi;
  j.q = h->q;
  j.key = h->key;
  j.i0 = (uint64_t)(h->T + 1);
  j.pb = h->pb;
  j.status = h->dstatus;
  return j;
}

// Decision phase of one block: one synchronisation for the row norms, the
// power-iteration values, the Ritz values and the sticky device status; then
// the first state-changing row is found, the rows before it are committed, the
// state is cut back to it and it is finished in FP64.
as_status block_finish(as_sketch* h, const BlockCtx& c, int64_t* used, bool* bad_row) {
  const int d = h->d, n2 = h->n2, r0 = c.r0, b = c.b, nbb = c.nbb;
  as_status st = AS_OK;
  *bad_row = false;
  AS_CUDA_TRY(cudaMemcpyAsync(h->h_buf, h->norm2, b * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  if (nbb > 0) {
    AS_CUDA_TRY(cudaMemcpyAsync(h->h_buf + b, h->pb.sig2, nbb * sizeof(double), cudaMemcpyDeviceToHost, h->s));
    AS_CUDA_TRY(cudaMemcpyAsync(h->h_buf + b + nbb, h->pb.ritz, 2 * nbb * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  }
  AS_CUDA_TRY(cudaMemcpyAsync(h->h_buf + b + 3 * nbb, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  {
    int ds = 0;
    std::memcpy(&ds, h->h_buf + b + 3 * nbb, sizeof(int));
    if (ds != 0) return (as_status)ds;
  }
  std::vector<double> a2(h->h_buf, h->h_buf + b);
  std::vector<double> sig2(h->h_buf + b, h->h_buf + b + nbb), ritz(h->h_buf + b + nbb, h->h_buf + b + 3 * nbb);
  int bb = b;
  for (int t = 0; t < b; ++t)
    if (!std::isfinite(a2[t])) { bb = t; *bad_row = true; break; }
  if (*bad_row) {
    AS_CUDA_TRY(cudaMemsetAsync(h->bad, 0, sizeof(int), h->s));
    st = launch_truncate(h->s, h->C, h->ldc, d, r0 + bb, r0 + b, h->G, n2);
    h->gf_valid = std::min(h->gf_valid, r0 + bb);
    if (st == AS_OK) st = tc_split_rows(h, r0 + bb, r0 + b);
    if (st != AS_OK) return st;
    if (bb == 0) { *used = 0; return AS_OK; }
  }
  // thresholds before each row (Algorithm 8)
  std::vector<double> Ft(bb), th(bb);
  double F = h->F;
  for (int t = 0; t < bb; ++t) {
    F += a2[t];
    Ft[t] = F;
    th[t] = (h->mode == AS_PERSISTENT) ? h->eps * F : h->theta;
  }
  const bool fills = (r0 + bb == n2);
  const int nb = std::min(nbb, fills ? bb - 1 : bb);
  // scan for the first state-changing row
  int tstar = -1, gate_known = -1;
  double sig2_star = 0.0;
  std::vector<char> gated((size_t)std::max(nb, 1), 0);
  for (int t = 0; t < nb; ++t) {
    const double theta = th[t];
    double s2 = sig2[t];
    const int64_t i = h->T + 1 + t;
    if (std::fabs(s2 - theta / 2.0) <= kTieBand * theta / 2.0 || theta == 0.0) {
      // tie band: the FP64 power iteration on the state seen by row t decides
      const int rsave = h->r;
      h->r = r0 + t + 1;
      st = pi_f64(h, i, &s2);
      h->r = rsave;
      if (st != AS_OK) return st;
    }
    const bool gate = s2 >= theta / 2.0 && s2 > 0.0;
    if (!gate) continue;
    gated[(size_t)t] = 1;
    const double r1 = ritz[2 * (size_t)t];
    if (r1 >= theta * (1.0 - kTieBand) || h->amp_r > 0) {  // a dump is possible (amplified: always)
      tstar = t;
      gate_known = 1;
      sig2_star = s2;
      break;
    }
    // gate passed, no component reaches theta: xi = 0, the state is unchanged
    h->st.gates++;
    h->st.si_runs++;
    if (h->cfg.flags & AS_TRACE_DECISIONS) {
      as_event ev{};
      ev.i = i; ev.sig2_pi = s2; ev.theta = theta; ev.j_stop = 1; ev.xi = 0;
      ev.ritz_1 = r1; ev.ritz_k = ritz[2 * (size_t)t + 1];
      h->trace.push_back(ev);
    }
  }
  // algorithmic work of the batch: the power iterations (k_PI products and the
  // Rayleigh quotient, 2 m_t^2 flop each) of the rows whose decision it gave,
  // and the k = 2 simultaneous iteration (q + 1 products of two columns) of the
  // gated rows that used it; rows after the first state-changing one were
  // speculation and are not counted
  const int bcol = (h->big && h->amp_r == 0 && tstar >= 0) ? batch_si_col(nbb, tstar) : -1;
  if (h->prof && c.batch_cls >= 0) {
    const int t_end = (tstar >= 0) ? tstar + 1 : nb;
    double w = 0.0;
    for (int t = 0; t < t_end; ++t) {
      const double m = (double)(r0 + t + 1);
      w += 2.0 * m * m * (double)(h->k_pi + 1);
    }
    for (int t = 0; t < t_end; ++t) {
      const bool gated_kept = (t < tstar || tstar < 0) ? gated[t] : (bcol >= 0);
      if (!gated_kept) continue;
      const double m = (double)(r0 + t + 1);
      w += 2.0 * m * m * 2.0 * (double)(h->q + 1);
    }
    h->prof->add_work(c.batch_cls, w);
  }
  if (tstar < 0 && fills) { tstar = bb - 1; gate_known = -1; }
  if (tstar < 0) {
    h->r = r0 + bb;
    h->T += bb;
    h->F = Ft[bb - 1];
    h->theta = th[bb - 1];
    *used = bb;
    h->bnext = std::min(h->bmax, h->bnext * 2);
    return AS_OK;
  }
  // commit rows 0..tstar, cut the speculative rows after it
  const int rnew = r0 + tstar + 1;
  if (rnew < r0 + bb) {
    st = launch_truncate(h->s, h->C, h->ldc, d, rnew, r0 + bb, h->G, n2);
    h->gf_valid = std::min(h->gf_valid, rnew);
    if (st == AS_OK) st = tc_split_rows(h, rnew, r0 + bb);
    if (st != AS_OK) return st;
  }
  h->r = rnew;
  h->T += tstar + 1;
  h->F = Ft[tstar];
  h->theta = th[tstar];
  *used = tstar + 1;
  h->bnext = std::max(8, std::min(h->bmax, 2 * (tstar + 1)));
  if (h->r == n2) {   // the buffer is full: FD shrink, then the row's decisions
    st = fd_shrink(h);
    if (st != AS_OK) return st;
    return finish_row(h, h->T, h->theta, -1, 0.0);
  }
  // large buffers reuse the batch's FP32-iterated basis for the k = 2 step (bcol)
  if (h->prof) h->prof->begin(PK_EVENT, h->s);
  st = finish_row(h, h->T, h->theta, gate_known, sig2_star, bcol, 3 * nbb);
  if (h->prof) h->prof->end(PK_EVENT, h->s, 0.0, 0.0);
  return st;
}

// ---- launch combiner: the FP32 batched iterations of many sketches --------
// Sketches updated together progress independently, each on its own host
// thread and stream; a block whose batched iterations would run the FP32
// persistent kernel hands its job to the device's combiner instead.  The
// combiner's thread launches whichever jobs are pending as one grouped
// cooperative launch (launch_batch_group) as soon as no other sketch of the
// update is in its launch phase (the only phase that can still add a job
// soon), or kCombineWindow after the first job arrived, whichever is earlier.
// No sketch waits for another's decision phase (the
// lockstep of earlier builds made every step wait for the slowest sketch's
// event rows).  Each job's result equals that of its own launch, so a
// sketch's results do not depend on the groups it landed in.
constexpr auto kCombineWindow = std::chrono::microseconds(40);

struct CombineReq {
  BatchJob job;
  as_sketch* h = nullptr;
  bool done = false;
  as_status st = AS_OK;
};

class Combiner {
 public:
  explicit Combiner(int dev) : dev_(dev) {}
  as_status start() {   // the calling thread's current device is left as it was
    int prev = 0;
    AS_CUDA_TRY(cudaGetDevice(&prev));
    AS_CUDA_TRY(cudaSetDevice(dev_));
    as_status st = AS_OK;
    if (cudaStreamCreateWithFlags(&gs_, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&gev_, cudaEventDisableTiming) != cudaSuccess) {
      as_note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
      st = AS_EDEVICE;
    }
    if (st == AS_OK) st = dalloc(&cnt_, 1);
    if (st == AS_OK) cap_ = batch_group_capacity();
    cudaSetDevice(prev);
    if (st != AS_OK) return st;
    th_ = std::thread([this] { loop(); });
    th_.detach();   // lives for the whole process, like the worker pool
    return AS_OK;
  }
  void enter() {
    std::lock_guard<std::mutex> lk(mu_);
    ++active_;
  }
  // a sketch's launch phase (which may end with a job for the combiner)
  void prep_begin() {
    std::lock_guard<std::mutex> lk(mu_);
    ++preparing_;
  }
  void prep_end() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      --preparing_;
    }
    cv_.notify_all();
  }
  void leave() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      --active_;
    }
    cv_.notify_all();
  }
  as_status submit(CombineReq* r) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (pending_.empty()) first_ = std::chrono::steady_clock::now();
      pending_.push_back(r);
      --preparing_;
    }
    cv_.notify_all();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return r->done; });
    return r->st;
  }

 private:
  void loop() {
    cudaSetDevice(dev_);
    std::vector<CombineReq*> batch;
    std::vector<BatchJob> jobs;
    for (;;) {
      batch.clear();
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return !pending_.empty(); });
        cv_.wait_until(lk, first_ + kCombineWindow,
                       [&] { return preparing_ == 0 || (int)pending_.size() >= active_; });
        int tiles = 0;
        size_t k = 0;
        for (; k < pending_.size() && batch.size() < 32; ++k) {
          const int t = batch_group_tiles(pending_[k]->job);
          if (!batch.empty() && (t <= 0 || tiles + t > cap_)) break;
          batch.push_back(pending_[k]);
          tiles += std::max(t, 0);
          if (t <= 0 || t > cap_) { ++k; break; }   // a job that cannot share a launch goes alone
        }
        pending_.erase(pending_.begin(), pending_.begin() + (long)k);
        if (!pending_.empty()) first_ = std::chrono::steady_clock::now();
      }
      launch(batch);
      {
        std::lock_guard<std::mutex> lk(mu_);
        for (CombineReq* r : batch) r->done = true;
      }
      done_cv_.notify_all();
    }
  }
  void launch(std::vector<CombineReq*>& batch) {
    as_status st = AS_ENOTSUP;
    if (batch.size() > 1) {
      jobs_.clear();
      for (CombineReq* r : batch) jobs_.push_back(r->job);
      cudaError_t e = cudaSuccess;
      for (CombineReq* r : batch)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(gs_, r->h->comb_ev, 0);
      st = (e == cudaSuccess) ? launch_batch_group(gs_, jobs_.data(), (int)jobs_.size(), cnt_) : as_from_cuda(e);
      if (st == AS_OK) {
        e = cudaEventRecord(gev_, gs_);
        for (CombineReq* r : batch) {
          if (e == cudaSuccess) e = cudaStreamWaitEvent(r->h->s, gev_, 0);
          r->h->st.grouped_batches++;
        }
        if (e != cudaSuccess) st = as_from_cuda(e);
        for (CombineReq* r : batch) r->st = st;
        return;
      }
    }
    // one job, or a group that did not fit: each job on its own sketch's stream
    for (CombineReq* r : batch) {
      const BatchJob& j = r->job;
      r->st = launch_batch_persist(r->h->s, j.Gf, j.n2, j.r0, j.nb, j.k_pi, j.q, j.key, j.i0, j.pb, j.status,
                                   r->h->prof);
    }
  }

  int dev_;
  cudaStream_t gs_ = nullptr;
  cudaEvent_t gev_ = nullptr;
  unsigned* cnt_ = nullptr;
  int cap_ = 0;
  std::thread th_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  std::vector<CombineReq*> pending_;
  std::vector<BatchJob> jobs_;
  std::chrono::steady_clock::time_point first_;
  int active_ = 0;
  int preparing_ = 0;   // sketches in a launch phase that has not handed over its job yet
};

std::mutex g_comb_mu;
std::map<int, Combiner*> g_comb;

// The device's combiner (made on first use; it lives for the whole process).
as_status combiner_for(int dev, Combiner** out) {
  std::lock_guard<std::mutex> lk(g_comb_mu);
  auto it = g_comb.find(dev);
  if (it != g_comb.end()) {
    *out = it->second;
    return AS_OK;
  }
  Combiner* c = new (std::nothrow) Combiner(dev);
  if (!c) return AS_ENOMEM;
  as_status st = c->start();
  if (st != AS_OK) return st;   // not kept (its thread did not start)
  g_comb[dev] = c;
  *out = c;
  return AS_OK;
}

// One block; with a combiner, FP32 batched iterations go through it.
as_status process_block(as_sketch* h, const float* src, int64_t navail, int64_t* used, bool* bad_row,
                        Combiner* comb = nullptr) {
  BlockCtx c;
  if (comb) comb->prep_begin();
  as_status st = block_prepare(h, src, navail, c, comb != nullptr);
  if (comb && (st != AS_OK || !c.deferred)) comb->prep_end();
  if (st != AS_OK) return st;
  if (c.deferred) {
    if (!h->comb_ev) AS_CUDA_TRY(cudaEventCreateWithFlags(&h->comb_ev, cudaEventDisableTiming));
    AS_CUDA_TRY(cudaEventRecord(h->comb_ev, h->s));
    CombineReq r;
    r.job = block_job(h, c);
    r.h = h;
    st = comb->submit(&r);   // ends the launch phase (prep_end) once the job is pending
    if (st != AS_OK) return st;
  }
  return block_finish(h, c, used, bad_row);
}

__global__ void add_f64_kernel(double* dst, const double* src, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] += src[e];
}

// The absorbed accumulator Bx (d x d FP64, zeroed) on first use.
as_status ensure_bx(as_sketch* h) {
  if (h->Bx) return AS_OK;
  as_status st = dalloc(&h->Bx, (size_t)h->d * h->d);
  if (st != AS_OK) return st;
  AS_CUDA_TRY(cudaMemsetAsync(h->Bx, 0, (size_t)h->d * h->d * sizeof(double), h->s));
  return AS_OK;
}

// B += Z Y + (Z Y)^T - Z (Y Z) Z^T for every snapshot of `src` taken at a
// row <= tmax (Algorithm 5), in time order, on stream st; the scratch
// of `scr` (xi x xi and d x xi) is grown as needed.
// The scratch of the snapshot-term products of scr, for snapshots of src.
as_status ensure_sx(const as_sketch* src, as_sketch* scr) {
  int ximax = 1;
  for (const Snap& sn : src->snaps) ximax = std::max(ximax, sn.xi);
  if (ximax <= scr->sx_cap) return AS_OK;
  if (scr->sx_yz) cudaFree(scr->sx_yz);
  if (scr->sx_t) cudaFree(scr->sx_t);
  scr->sx_yz = scr->sx_t = nullptr;
  scr->sx_cap = 0;
  as_status st2 = dalloc(&scr->sx_yz, (size_t)ximax * ximax);
  if (st2 == AS_OK) st2 = dalloc(&scr->sx_t, (size_t)scr->d * ximax);
  if (st2 != AS_OK) return st2;
  scr->sx_cap = ximax;
  return AS_OK;
}

as_status add_snapshot_terms(const as_sketch* src, int64_t tmax, double* B, as_sketch* scr, cudaStream_t st,
                             int64_t tmin_excl = INT64_MIN) {
  const int d = src->d;
  {
    as_status st2 = ensure_sx(src, scr);
    if (st2 != AS_OK) return st2;
  }
  double* YZ = scr->sx_yz;
  double* T = scr->sx_t;
  as_status st2 = AS_OK;
  for (const Snap& sn : src->snaps) {
    if (sn.t > tmax) break;   // the queue is in time order
    if (sn.t <= tmin_excl) continue;
    const float* Z = src->arena + sn.off;
    const float* Y = Z + (size_t)d * sn.xi;
    const int xi = sn.xi;
    if ((st2 = gemm_strided<float, float, double>(st, d, d, xi, Z, xi, 1, Y, d, 1, B, d, 1, 1.0, 1.0)) != AS_OK) break;
    if ((st2 = gemm_strided<float, float, double>(st, d, d, xi, Z, xi, 1, Y, d, 1, B, 1, d, 1.0, 1.0)) != AS_OK) break;
    if ((st2 = gemm_strided<float, float, double>(st, xi, xi, d, Y, d, 1, Z, xi, 1, YZ, xi, 1, 1.0, 0.0)) != AS_OK) break;
    if ((st2 = gemm_strided<float, double, double>(st, d, xi, xi, Z, xi, 1, YZ, xi, 1, T, xi, 1, 1.0, 0.0)) != AS_OK) break;
    if ((st2 = gemm_strided<double, float, double>(st, d, d, xi, T, xi, 1, Z, 1, xi, B, d, 1, -1.0, 1.0)) != AS_OK) break;
  }
  return st2;
}

// The matrix B of Algorithm 5 (before its eigendecomposition) with lb = 0, ub = t: the residual C_t only at the
// current time (t = T; older residuals are not stored) plus the snapshot
// terms with t_j <= t, plus (current time only) the absorbed terms Bx.
as_status build_query_gram(as_sketch* h, int64_t t, double* B) {
  const int d = h->d;
  as_status st = AS_OK;
  AS_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)d * d * sizeof(double), h->s));
  if (t == h->T && h->r > 0) {
    st = gemm_strided<float, float, double>(h->s, d, d, h->r, h->C, 1, h->ldc, h->C, h->ldc, 1, B, d, 1, 1.0, 0.0);
    if (st != AS_OK) return st;
  }
  st = add_snapshot_terms(h, t, B, h, h->s);
  if (st == AS_OK && t == h->T && h->Bx) {
    add_f64_kernel<<<256, 256, 0, h->s>>>(B, h->Bx, (size_t)d * d); count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
  }
  cudaStreamSynchronize(h->s);
  return st;
}

// Eigendecomposition of the device matrix B (d x d FP64, destroyed) and the
// eigen-shrink of Algorithm 5: the l x d sketch to out (host or device,
// row stride ldo).  Synchronises.
as_status eig_shrink_to(as_sketch* h, double* B, float* out, int64_t ldo) {
  const int d = h->d, ell = h->ell;
  double *lam = nullptr, *V = nullptr, *w = nullptr;
  float* o = nullptr;
  const bool big_q = d > 256;
  as_status st = dalloc(&lam, (size_t)d);
  if (st == AS_OK) st = dalloc(&V, (size_t)d * ell);
  if (st == AS_OK) st = dalloc(&w, big_q ? eig_large_work_doubles(d, ell) : eig_work_doubles(d, ell));
  if (st == AS_OK) st = dalloc(&o, (size_t)ell * d);
  if (st == AS_OK)
    st = big_q ? launch_eig_large(h->s, d, B, d, ell, lam, V, ell, w, nullptr, h->dstatus)
               : launch_eig(h->s, d, B, d, ell, lam, V, ell, w);
  if (st == AS_OK) st = launch_shrink_rows(h->s, d, ell, lam, V, ell, o, d);
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpy2DAsync(out, (size_t)ldo * sizeof(float), o, (size_t)d * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)ell, cudaMemcpyDefault, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) {
    as_status ds = sync_status(h);
    if (ds != AS_OK) st = ds;
  }
  cudaFree(lam); cudaFree(V); cudaFree(w); cudaFree(o);
  return st;
}

// The low-rank route of Algorithm 5 (lowrank.cu explains the algebra): B_hat
// of time t to the device buffer o (l x d, row-major).  *used = false (and
// nothing written) when the route does not apply: merged terms present, the
// stacked factor rows r_F above 3d/4, or AS_QUERY_DENSE.
as_status query_lowrank(as_sketch* h, int64_t t, float* o, bool* used) {
  *used = false;
  const int d = h->d, ell = h->ell;
  if (h->cfg.flags & AS_QUERY_DENSE) return AS_OK;
  if (t == h->T && h->Bx) return AS_OK;
  const int rc = (t == h->T) ? h->r : 0;
  int64_t rf64 = rc;
  for (const Snap& sn : h->snaps) {
    if (sn.t > t) break;
    rf64 += 2 * (int64_t)sn.xi;
  }
  if (rf64 < 1 || 4 * rf64 > 3 * (int64_t)d) return AS_OK;
  const int rF = (int)rf64;
  float* F = nullptr;
  double *W = nullptr, *Ws = nullptr, *Hs = nullptr, *lw = nullptr, *U = nullptr, *ew = nullptr, *T = nullptr;
  double *K = nullptr, *mu = nullptr, *Uk = nullptr, *P = nullptr, *V = nullptr, *lam = nullptr;
  int4* kind = nullptr;
  const bool big = rF > 256;
  as_status st = dalloc(&F, (size_t)rF * d);
  if (st == AS_OK) st = dalloc(&W, (size_t)rF * rF);
  if (st == AS_OK) st = dalloc(&Ws, (size_t)rF * rF);
  if (st == AS_OK) st = dalloc(&Hs, (size_t)rF * rF);
  if (st == AS_OK) st = dalloc(&lw, (size_t)rF);
  if (st == AS_OK) st = dalloc(&U, (size_t)rF * rF);
  if (st == AS_OK) st = dalloc(&ew, big ? eig_large_work_doubles(rF, rF) : eig_work_doubles(rF, rF));
  if (st == AS_OK) st = dalloc(&T, (size_t)rF * rF);
  if (st == AS_OK) st = dalloc(&kind, (size_t)rF);
  std::vector<int4> hk((size_t)rF);
  // F = [C; Z_1^T; Y_1; ...] (FP32, ld d) and the row kinds
  int row = 0;
  if (st == AS_OK && rc > 0) {
    cudaError_t e = cudaMemcpy2DAsync(F, (size_t)d * sizeof(float), h->C, (size_t)h->ldc * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)rc, cudaMemcpyDeviceToDevice, h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
    for (; row < rc; ++row) hk[(size_t)row] = make_int4(0, 0, 0, 0);
  }
  for (const Snap& sn : h->snaps) {
    if (st != AS_OK || sn.t > t) break;
    const float* Z = h->arena + sn.off;
    const float* Y = Z + (size_t)d * sn.xi;
    st = launch_transpose_f32(h->s, Z, d, sn.xi, F + (size_t)row * d, d);
    if (st != AS_OK) break;
    cudaError_t e = cudaMemcpyAsync(F + (size_t)(row + sn.xi) * d, Y, (size_t)sn.xi * d * sizeof(float),
                                    cudaMemcpyDeviceToDevice, h->s);
    if (e != cudaSuccess) { st = as_from_cuda(e); break; }
    for (int a = 0; a < sn.xi; ++a) {
      hk[(size_t)(row + a)] = make_int4(1, row, sn.xi, 0);
      hk[(size_t)(row + sn.xi + a)] = make_int4(2, row, sn.xi, 0);
    }
    row += 2 * sn.xi;
  }
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpyAsync(kind, hk.data(), (size_t)rF * sizeof(int4), cudaMemcpyHostToDevice, h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  // W = F F^T in FP64 (F's FP32 values are exact; FP32 partial sums would leave
  // noise of about 1e-7 in W', above the rank cutoff), scaled; H' from it
  if (st == AS_OK) {
    double* F64 = nullptr;
    st = dalloc(&F64, (size_t)rF * d);
    if (st == AS_OK) st = launch_f32_to_f64(h->s, F, (size_t)rF * d, F64);
    if (st == AS_OK)
      st = gemm_strided<double, double, double>(h->s, rF, rF, d, F64, d, 1, F64, 1, d, W, rF, 1, 1.0, 0.0);
    if (F64) {
      cudaStreamSynchronize(h->s);
      cudaFree(F64);
    }
  }
  if (st == AS_OK) st = launch_lr_scale(h->s, W, rF, kind, Ws, Hs);
  // W' = U L U^T (all rF pairs), then the numerical rank r'
  if (st == AS_OK)
    st = big ? launch_eig_large(h->s, rF, Ws, rF, rF, lw, U, rF, ew, nullptr, h->dstatus)
             : launch_eig(h->s, rF, Ws, rF, rF, lw, U, rF, ew);
  std::vector<double> hl((size_t)rF);
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpyAsync(hl.data(), lw, (size_t)rF * sizeof(double), cudaMemcpyDeviceToHost, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) st = sync_status(h);
  int rr = 0;
  if (st == AS_OK && hl[0] > 0.0) {
    const double cut = 1e-10 * hl[0];
    while (rr < rF && hl[(size_t)rr] > cut) ++rr;
  }
  const int lp = std::min(ell, rr);
  if (st == AS_OK) st = dalloc(&V, (size_t)d * ell);
  if (st == AS_OK) st = dalloc(&lam, (size_t)ell);
  if (st == AS_OK) {
    cudaError_t e = cudaMemsetAsync(V, 0, (size_t)d * ell * sizeof(double), h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK && rr > 0) {
    const bool bigk = rr > 256;
    double* ek = nullptr;
    st = dalloc(&K, (size_t)rr * rr);
    if (st == AS_OK) st = dalloc(&mu, (size_t)lp);
    if (st == AS_OK) st = dalloc(&Uk, (size_t)rr * lp);
    if (st == AS_OK) st = dalloc(&P, (size_t)rF * lp);
    if (st == AS_OK) st = dalloc(&ek, bigk ? eig_large_work_doubles(rr, lp) : eig_work_doubles(rr, lp));
    // T = H' U_r (rF x r'), K0 = U_r^T T, K = L^1/2 sym(K0) L^1/2
    if (st == AS_OK)
      st = gemm_strided<double, double, double>(h->s, rF, rr, rF, Hs, rF, 1, U, rF, 1, T, rr, 1, 1.0, 0.0);
    if (st == AS_OK)
      st = gemm_strided<double, double, double>(h->s, rr, rr, rF, U, 1, rF, T, rr, 1, Ws, rr, 1, 1.0, 0.0);
    if (st == AS_OK) st = launch_lr_core(h->s, Ws, rr, lw, rr, K);
    if (st == AS_OK)
      st = bigk ? launch_eig_large(h->s, rr, K, rr, lp, mu, Uk, lp, ek, nullptr, h->dstatus)
                : launch_eig(h->s, rr, K, rr, lp, mu, Uk, lp, ek);
    // E = D U_r L_r^-1/2 U_k, V = F^T E
    if (st == AS_OK) st = launch_lr_colscale(h->s, U, rF, rF, lw, rr);
    if (st == AS_OK)
      st = gemm_strided<double, double, double>(h->s, rF, lp, rr, U, rF, 1, Uk, lp, 1, P, lp, 1, 1.0, 0.0);
    if (st == AS_OK) st = launch_lr_rowscale(h->s, W, rF, P, lp);
    if (st == AS_OK)
      st = gemm_strided<float, double, double>(h->s, d, lp, rF, F, 1, d, P, lp, 1, V, ell, 1, 1.0, 0.0);
    if (st == AS_OK) st = launch_lr_lambda(h->s, mu, lp, ell, lam);
    if (ek) cudaFree(ek);
  } else if (st == AS_OK) {
    cudaError_t e = cudaMemsetAsync(lam, 0, (size_t)ell * sizeof(double), h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) st = launch_shrink_rows(h->s, d, ell, lam, V, ell, o, d);
  if (st == AS_OK) {
    cudaError_t e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) st = sync_status(h);
  void* ptrs[] = {F, W, Ws, Hs, lw, U, ew, T, K, mu, Uk, P, V, lam, kind};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (st == AS_OK) *used = true;
  return st;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---- library-internal access for the runtimes built on sketches (sliding.cu)
namespace as {

cudaStream_t sk_stream(const as_sketch* h) { return h->s; }
int sk_device(const as_sketch* h) { return h->dev; }
int64_t sk_device_bytes(const as_sketch* h) { return (int64_t)h->dev_bytes; }
int64_t sk_rows(const as_sketch* h) { return h->T; }
int sk_snap_count(const as_sketch* h) { return (int)h->snaps.size(); }
int64_t sk_snap_t(const as_sketch* h, int k) { return h->snaps[(size_t)k].t; }

// B = C^T C (the current residual) + the snapshot terms with t > lb (the
// sketch's own row times), on the sketch's stream; B is d x d FP64 device.
as_status sk_window_gram(as_sketch* h, int64_t lb, double* B) {
  const int d = h->d;
  AS_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)d * d * sizeof(double), h->s));
  as_status st = AS_OK;
  if (h->r > 0)
    st = gemm_strided<float, float, double>(h->s, d, d, h->r, h->C, 1, h->ldc, h->C, h->ldc, 1, B, d, 1, 1.0, 0.0);
  if (st == AS_OK) st = add_snapshot_terms(h, INT64_MAX, B, h, h->s, lb);
  return st;
}

// B += R^T R for the k rows of R (device FP32, row stride ld).
as_status sk_add_rows_gram(as_sketch* h, const float* R, int k, int64_t ld, double* B) {
  if (k <= 0) return AS_OK;
  const int d = h->d;
  return gemm_strided<float, float, double>(h->s, d, d, k, R, 1, ld, R, ld, 1, B, d, 1, 1.0, 1.0);
}

// Remove the `count` oldest snapshots; the arena is compacted once the dropped
// prefix is at least as long as the live part (the copy then cannot overlap).
as_status sk_drop_front(as_sketch* h, int count) {
  count = std::min(count, (int)h->snaps.size());
  if (count <= 0) return AS_OK;
  for (int k = 0; k < count; ++k) h->st.snapshot_rank -= h->snaps[(size_t)k].xi;
  h->snaps.erase(h->snaps.begin(), h->snaps.begin() + count);
  if (h->snaps.empty()) {
    h->arena_used = 0;
    return AS_OK;
  }
  const size_t head = h->snaps.front().off;
  const size_t live = h->arena_used - head;
  if (head >= live) {
    AS_CUDA_TRY(cudaMemcpyAsync(h->arena, h->arena + head, live * sizeof(float), cudaMemcpyDeviceToDevice, h->s));
    for (Snap& sn : h->snaps) sn.off -= head;
    h->arena_used = live;
  }
  return AS_OK;
}

as_status sk_eig_shrink(as_sketch* h, double* B, float* out, int64_t ldo) { return eig_shrink_to(h, B, out, ldo); }

}  // namespace as


namespace {
// The calling thread's last failed CUDA call, and the last one of any thread
// (runtimes such as the server run sketches on worker threads).
thread_local char g_last_error[192] = "";
char g_last_error_any[192] = "";
std::mutex g_last_error_mu;
std::mutex g_smem_mu;
std::map<std::pair<const void*, int>, size_t> g_smem_limit;   // (kernel, device) -> limit set
}

void as_note_cuda_error(cudaError_t e, const char* file, int line) {
  const char* base = std::strrchr(file, '/');
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", cudaGetErrorName(e), base ? base + 1 : file, line);
  std::lock_guard<std::mutex> lk(g_last_error_mu);
  std::memcpy(g_last_error_any, g_last_error, sizeof(g_last_error));
}

cudaError_t as_raise_smem_limit(const void* fn, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& cur = g_smem_limit[{fn, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}


// Validate a configuration and fill its defaults; the amplification counts of
// Algorithm 7 come back in amp_r, amp_s (0 when off).
static as_status normalize_config(as_config& c, int& amp_r, int& amp_s) {
  if (c.d < 2) return AS_EINVAL;
  if (!(c.eps >= 0.0) || std::isinf(c.eps)) return AS_EINVAL;
  if (c.ell == 0) {
    if (c.eps <= 0.0) return AS_EINVAL;
    c.ell = (int32_t)std::ceil(2.0 / c.eps);  // Algorithm 3
  }
  if (c.ell < 1 || 2 * (int64_t)c.ell > c.d) return AS_EINVAL;
  if (c.eps == 0.0) c.eps = 2.0 / c.ell;
  if (c.mode == AS_SLIDING) return AS_ENOTSUP;
  if (c.mode != AS_PERSISTENT && c.mode != AS_FIXED_THETA && c.mode != AS_SITE && c.mode != AS_COORDINATOR)
    return AS_EINVAL;
  if ((c.mode == AS_FIXED_THETA || c.mode == AS_SITE) && !(c.theta >= 0.0)) return AS_EINVAL;
  if (c.prec != AS_FP32_PLAIN && c.prec != AS_BF16 && c.prec != AS_BF16X3 && c.prec != AS_BF16X6) return AS_EINVAL;
  if (c.prec != AS_FP32_PLAIN && !umma_available()) return AS_ENOTSUP;
  if (c.eps_si == 0.0) c.eps_si = 0.4;
  if (!(c.eps_si > 0.0 && c.eps_si < 1.0)) return AS_EINVAL;
  if (c.k_pi < 0 || c.q_si < 0) return AS_EINVAL;
  if (c.k_pi == 0) c.k_pi = ceil_log2(c.d) + 1;                              // Corollary 1
  if (c.q_si == 0) c.q_si = (int32_t)std::ceil(std::log((double)c.d) / c.eps_si);  // Theta(log d / eps_SI)
  // Algorithm 7: r = ceil(log_100(2/delta)) SIs, s = ceil(2 log_3(2/delta))
  // estimates each; r <= 15 and s <= 63 keep the trace's 4-bit choices and the
  // Philox sub-indices 64 h + g of the estimates distinct
  amp_r = amp_s = 0;
  if (c.delta != 0.0) {
    if (!(c.delta > 0.0 && c.delta < 1.0)) return AS_EINVAL;
    const double lg = std::log(2.0 / c.delta);
    amp_r = std::max(1, (int)std::ceil(lg / std::log(100.0)));
    amp_s = std::max(1, (int)std::ceil(2.0 * lg / std::log(3.0)));
    if (amp_r > 15 || amp_s > 63) return AS_EINVAL;
  }
  return AS_OK;
}

// The sketch's shape and control fields from a normalised configuration.
static void init_fields(as_sketch* h, const as_config& c, int amp_r, int amp_s, void* cuda_stream) {
  h->cfg = c;
  h->d = c.d;
  h->ell = c.ell;
  h->n2 = 2 * c.ell;
  h->ldc = (c.d + 63) / 64 * 64;
  h->eps = c.eps;
  h->eps_si = c.eps_si;
  h->k_pi = c.k_pi;
  h->q = c.q_si;
  h->amp_r = amp_r;
  h->amp_s = amp_s;
  h->q_amp = (int)std::ceil(std::log((double)c.d) / 0.2);
  h->mode = c.mode;
  h->theta = (c.mode == AS_FIXED_THETA || c.mode == AS_SITE) ? c.theta : 0.0;
  const int mn = std::min(c.ell, c.d);
  h->jmax = (mn > 1) ? ceil_log2(mn) : 0;
  h->s = (cudaStream_t)cuda_stream;
  h->key = Key{c.seed, c.stream_id};
  h->stage_rows = 256;
  h->big = h->n2 >= kMultiRowMin;
  h->big_eig = h->n2 >= kEigLargeMin;
  h->bmax = 64;
  h->bnext = 64;
}

// Allocate the device state of a sketch whose fields are set (init_fields);
// with dry = true nothing is allocated and only the byte count is returned.
static as_status alloc_state(as_sketch* h, bool dry, size_t* out_bytes) {
  const int n2 = h->n2, ell = h->ell, kmax = ell, bmax = h->bmax;
  size_t bytes = 0;
  as_status st = AS_OK;
#define ALLOC(ptr, n)                                          \
  do {                                                         \
    if (st == AS_OK) {                                         \
      if (!dry) st = dalloc(&(ptr), (n));                      \
      bytes += (size_t)(n) * sizeof(*(ptr));                   \
    }                                                          \
  } while (0)
  ALLOC(h->C, (size_t)n2 * h->ldc);
  ALLOC(h->Cnew, (size_t)n2 * h->ldc);
  ALLOC(h->Wfd, (size_t)ell * n2);
  ALLOC(h->stage, (size_t)h->stage_rows * h->d);
  ALLOC(h->G, (size_t)n2 * n2);
  ALLOC(h->Gtmp, (size_t)n2 * n2);
  ALLOC(h->lam, (size_t)n2);
  ALLOC(h->U, (size_t)n2 * ell);
  ALLOC(h->eigw, h->big_eig ? eig_large_work_doubles(n2, ell) : eig_work_doubles(n2, ell));
  ALLOC(h->scal, 1024);
  ALLOC(h->bad, 1);
  ALLOC(h->dstatus, 1);
  ALLOC(h->zero, 1);
  ALLOC(h->x64, (size_t)n2);
  ALLOC(h->y64, (size_t)n2);
  ALLOC(h->norm2, (size_t)bmax);
  ALLOC(h->Gf, (size_t)n2 * n2);
  h->bb.max_splits = 16;
  h->p_cap = std::max({(size_t)h->bb.max_splits * n2 * 3 * bmax, (size_t)64 * bmax * n2,
                       (size_t)16 * ell * ell});
  ALLOC(h->bb.P, h->p_cap);
  h->pb.ycols = batch_persist_ycols(bmax);
  h->pb.ldy = (n2 + 31) / 32 * 32;
  h->pb.ybuf = (long long)h->pb.ldy * (long long)h->pb.ycols;
  h->pb.bmax = bmax;
  ALLOC(h->pb.Y, 2 * (size_t)h->pb.ybuf);
  ALLOC(h->pb.X, (size_t)n2 * h->pb.ycols);
  ALLOC(h->pb.part, batch_persist_part_floats(bmax));
  ALLOC(h->pb.cnt, 1);
  ALLOC(h->pb.sig2, (size_t)bmax);
  ALLOC(h->pb.ritz, (size_t)2 * bmax);
  ALLOC(h->si.Y, (size_t)n2 * kmax);
  ALLOC(h->si.GY, (size_t)n2 * kmax);
  ALLOC(h->si.S, (size_t)kmax * kmax);
  ALLOC(h->si.V, (size_t)kmax * kmax);
  ALLOC(h->si.eigw, eig_work_doubles(kmax, kmax));
  ALLOC(h->si.ritz, (size_t)kmax);
  ALLOC(h->si.WU, (size_t)n2 * kmax);
  ALLOC(h->si.GWU, (size_t)n2 * kmax);
  ALLOC(h->si.tmp, (size_t)n2 * kmax + 3 * (size_t)kmax * kmax + kmax);
  if (st == AS_OK && h->cfg.prec != AS_FP32_PLAIN) {
    h->tc = true;
    h->dpass = (h->cfg.prec == AS_BF16X6) ? 6 : (h->cfg.prec == AS_BF16X3) ? 3 : 1;
    h->n2p = (n2 + 63) / 64 * 64;
    const int rp = std::max(256, std::max(n2, std::max(3 * bmax, ell)));
    h->rows_pad = rp;
    const size_t cN = (size_t)std::max(rp, n2) * h->ldc, ctN = (size_t)std::max(h->d, 256) * h->n2p;
    const size_t wN = (size_t)std::max(ell, 256) * h->n2p;
    ALLOC(h->Chi, cN); ALLOC(h->Clo, cN); ALLOC(h->Cthi, ctN); ALLOC(h->Ctlo, ctN);
    ALLOC(h->Wh, wN); ALLOC(h->Wl, wN);
    if (h->dpass == 6) { ALLOC(h->Cl2, cN); ALLOC(h->Ctl2, ctN); ALLOC(h->Wl2, wN); }
    if (n2 >= 256) {   // the tcgen05 batched iterations: BF16 levels of G and of the batch vectors
      h->tcb = true;
      h->tb.ldg = h->n2p;
      h->tb.glevel = (long long)h->n2p * h->n2p;
      h->tb.ldyb = (n2 + 127) / 128 * 128;
      h->tb.yblevel = 2LL * (long long)h->pb.ycols * h->tb.ldyb;
      ALLOC(h->tb.Gb, 3 * (size_t)h->tb.glevel);
      ALLOC(h->tb.Yb, 3 * (size_t)h->tb.yblevel);
      ALLOC(h->tb.part, batch_tc_part_floats(n2, (int)h->pb.ycols));
    }
    if (dry) {
      *out_bytes = bytes;
      return st;
    }
    __nv_bfloat16* bz[] = {h->Chi, h->Clo, h->Cthi, h->Ctlo, h->Wh, h->Wl, h->Cl2, h->Ctl2, h->Wl2, h->tb.Gb, h->tb.Yb};
    const size_t bn[] = {cN, cN, ctN, ctN, wN, wN, cN, ctN, wN, 3 * (size_t)h->tb.glevel, 3 * (size_t)h->tb.yblevel};
    for (int t = 0; t < 11 && st == AS_OK; ++t)
      if (bz[t] && cudaMemsetAsync(bz[t], 0, bn[t] * sizeof(__nv_bfloat16), h->s) != cudaSuccess) st = AS_EDEVICE;
    const int cr = (int)(cN / h->ldc);
    // level maps; a missing third level repeats the second (never read then)
    auto mk = [&](UmmaOperand& o, __nv_bfloat16* l0, __nv_bfloat16* l1, __nv_bfloat16* l2, int rows, int kdim,
                  long long ld, int box) {
      if (st != AS_OK) return;
      st = umma_make_map(&o.m[0], l0, rows, kdim, ld, box);
      if (st == AS_OK) st = umma_make_map(&o.m[1], l1, rows, kdim, ld, box);
      if (st == AS_OK) st = umma_make_map(&o.m[2], l2 ? l2 : l1, rows, kdim, ld, box);
    };
    mk(h->mCA, h->Chi, h->Clo, h->Cl2, cr, h->ldc, h->ldc, 128);
    mk(h->mCB64, h->Chi, h->Clo, h->Cl2, cr, h->ldc, h->ldc, 64);
    mk(h->mCB256, h->Chi, h->Clo, h->Cl2, cr, h->ldc, h->ldc, 256);
    mk(h->mWA, h->Wh, h->Wl, h->Wl2, (int)(wN / h->n2p), h->n2p, h->n2p, 128);
    mk(h->mCtB, h->Cthi, h->Ctlo, h->Ctl2, (int)(ctN / h->n2p), h->n2p, h->n2p, 64);
    if (h->tcb)
      mk(h->tb.mG, h->tb.Gb, h->tb.Gb + h->tb.glevel, h->tb.Gb + 2 * h->tb.glevel, h->n2p, h->n2p, h->n2p, 128);
  }
#undef ALLOC
  *out_bytes = bytes;
  return st;
}

extern "C" {

const char* as_last_error(void) {
  if (!g_last_error[0]) {
    std::lock_guard<std::mutex> lk(g_last_error_mu);
    std::memcpy(g_last_error, g_last_error_any, sizeof(g_last_error));
  }
  return g_last_error;
}

as_status as_inject_alloc_failure(int32_t after) {
  if (after < -1) return AS_EINVAL;
  g_fail_after.store(after);
  return AS_OK;
}

const char* as_status_str(as_status s) {
  switch (s) {
    case AS_OK: return "AS_OK";
    case AS_EINVAL: return "AS_EINVAL";
    case AS_ENOMEM: return "AS_ENOMEM";
    case AS_EDEVICE: return "AS_EDEVICE";
    case AS_ENUMERIC: return "AS_ENUMERIC";
    case AS_ETIMEOUT: return "AS_ETIMEOUT";
    case AS_EBUSY: return "AS_EBUSY";
    case AS_ENOTSUP: return "AS_ENOTSUP";
  }
  return "AS_UNKNOWN";
}

as_status sketch_create(const as_config* cfg, void* cuda_stream, as_sketch** out) {
  if (!cfg || !out) return AS_EINVAL;
  *out = nullptr;
  as_config c = *cfg;
  int amp_r = 0, amp_s = 0;
  as_status st0 = normalize_config(c, amp_r, amp_s);
  if (st0 != AS_OK) return st0;
  as_sketch* h = new (std::nothrow) as_sketch();
  if (!h) return AS_ENOMEM;
  init_fields(h, c, amp_r, amp_s, cuda_stream);
  if (cudaGetDevice(&h->dev) != cudaSuccess) {
    as_note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
    delete h;
    return AS_EDEVICE;
  }
  const int n2 = h->n2, bmax = h->bmax;
  size_t bytes = 0;
  as_status st = alloc_state(h, false, &bytes);
  if (st == AS_OK && cudaMallocHost((void**)&h->h_buf, (size_t)(4 * std::max(n2, bmax) + 64) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->h_buf = nullptr;
    st = AS_ENOMEM;
  }
  if (st == AS_OK) {
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemsetAsync(h->C, 0, (size_t)n2 * h->ldc * sizeof(float), h->s);
    e = e ? e : cudaMemsetAsync(h->G, 0, (size_t)n2 * n2 * sizeof(double), h->s);
    e = e ? e : cudaMemsetAsync(h->bad, 0, sizeof(int), h->s);
    e = e ? e : cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->s);
    e = e ? e : cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st != AS_OK) {
    free_all(h);
    delete h;
    return st;
  }
  h->dev_bytes = bytes;
  if (c.flags & AS_PROFILE) h->prof = new (std::nothrow) EventProf();
  h->st.d = h->d;
  h->st.ell = h->ell;
  *out = h;
  return AS_OK;
}

as_status sketch_footprint(const as_config* cfg, int64_t snapshot_rank, int64_t* bytes) {
  if (!cfg || !bytes || snapshot_rank < 0) return AS_EINVAL;
  as_config c = *cfg;
  int amp_r = 0, amp_s = 0;
  as_status st = normalize_config(c, amp_r, amp_s);
  if (st != AS_OK) return st;
  as_sketch t;
  init_fields(&t, c, amp_r, amp_s, nullptr);
  size_t b = 0;
  st = alloc_state(&t, true, &b);
  if (st != AS_OK) return st;
  b += dwork_max(&t) * sizeof(double) + prb_max(&t) * sizeof(float);
  b += (size_t)2 * t.d * (size_t)snapshot_rank * sizeof(float);
  *bytes = (int64_t)b;
  return AS_OK;
}

as_status sketch_reserve(as_sketch* h, int64_t snapshot_rank) {
  if (!h || snapshot_rank < 0) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
  if (!lk.owns_lock()) return AS_EBUSY;
  as_status st = ensure_dwork(h, dwork_max(h));
  if (st == AS_OK && h->tc) st = ensure_prb(h, prb_max(h));
  if (st == AS_OK && snapshot_rank > 0) st = arena_reserve(h, (size_t)2 * h->d * (size_t)snapshot_rank, true);
  return st;
}

// sketch_update, with the FP32 batched iterations going through the device's
// launch combiner when comb is given.
static as_status update_rows(as_sketch* h, const float* rows, int64_t n, int64_t ld, Combiner* comb) {
  if (!h) return AS_EINVAL;
  if (h->mode == AS_COORDINATOR) return AS_EINVAL;   // a coordinator only receives
  if (n == 0) return AS_OK;
  if (!rows || n < 0 || ld < h->d) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
  if (!lk.owns_lock()) return AS_EBUSY;
  const bool dev = is_device_ptr(rows);
  as_status st = AS_OK;
  for (int64_t t0 = 0; t0 < n && st == AS_OK; t0 += h->stage_rows) {
    const int64_t nb = std::min<int64_t>(h->stage_rows, n - t0);
    const float* src = rows + t0 * ld;
    const float* base = src;
    int64_t ldb = ld;
    if (!dev) {
      cudaError_t e = cudaMemcpy2DAsync(h->stage, (size_t)h->d * sizeof(float), src, (size_t)ld * sizeof(float),
                                        (size_t)h->d * sizeof(float), (size_t)nb, cudaMemcpyHostToDevice, h->s);
      if (e != cudaSuccess) return as_from_cuda(e);
      base = h->stage;
      ldb = h->d;
    }
    if (ldb != h->d) {
      // rows with a padded stride: compact them into the staging buffer
      cudaError_t e = cudaMemcpy2DAsync(h->stage, (size_t)h->d * sizeof(float), base, (size_t)ldb * sizeof(float),
                                        (size_t)h->d * sizeof(float), (size_t)nb, cudaMemcpyDeviceToDevice, h->s);
      if (e != cudaSuccess) return as_from_cuda(e);
      base = h->stage;
    }
    int64_t done = 0;
    while (done < nb && st == AS_OK) {
      int64_t used = 0;
      bool bad = false;
      st = process_block(h, base + done * h->d, nb - done, &used, &bad, comb);
      done += used;
      if (st == AS_OK && bad) st = AS_EINVAL;
    }
  }
  if (st == AS_OK) {
    as_status ds = sync_status(h);
    if (ds != AS_OK) st = ds;
  }
  return st;
}

as_status sketch_update(as_sketch* h, const float* rows, int64_t n, int64_t ld) {
  return update_rows(h, rows, n, ld, nullptr);
}



as_status sketch_query_gram(as_sketch* h, int64_t t, double* out) {
  if (!h || !out) return AS_EINVAL;
  if (t == -1) t = h->T;
  if (t < 0 || t > h->T) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
  if (!lk.owns_lock()) return AS_EBUSY;
  double* B = nullptr;
  as_status st = dalloc(&B, (size_t)h->d * h->d);
  if (st != AS_OK) return st;
  st = build_query_gram(h, t, B);
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpy(out, B, (size_t)h->d * h->d * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  cudaFree(B);
  return st;
}

as_status sketch_query(as_sketch* h, int64_t t, float* out, int64_t ldo, int32_t* rows_out) {
  if (!h || !out || ldo < h->d) return AS_EINVAL;
  if (t == -1) t = h->T;
  if (t < 0 || t > h->T) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
  if (!lk.owns_lock()) return AS_EBUSY;
  const int d = h->d, ell = h->ell;
  double *B = nullptr, *lam = nullptr, *V = nullptr, *w = nullptr;
  float* o = nullptr;
  as_status st = dalloc(&o, (size_t)ell * d);
  bool low = false;
  if (st == AS_OK) st = query_lowrank(h, t, o, &low);
  if (st == AS_OK && !low) {   // the dense route: B (d x d), its eigendecomposition, the shrink by lambda_l
    const bool big_q = d > 256;
    st = dalloc(&B, (size_t)d * d);
    if (st == AS_OK) st = dalloc(&lam, (size_t)d);
    if (st == AS_OK) st = dalloc(&V, (size_t)d * ell);
    if (st == AS_OK) st = dalloc(&w, big_q ? eig_large_work_doubles(d, ell) : eig_work_doubles(d, ell));
    if (st == AS_OK) st = build_query_gram(h, t, B);
    if (st == AS_OK)
      st = big_q ? launch_eig_large(h->s, d, B, d, ell, lam, V, ell, w, nullptr, h->dstatus)
                 : launch_eig(h->s, d, B, d, ell, lam, V, ell, w);
    if (st == AS_OK) st = launch_shrink_rows(h->s, d, ell, lam, V, ell, o, d);
  }
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpy2DAsync(out, (size_t)ldo * sizeof(float), o, (size_t)d * sizeof(float),
                                      (size_t)d * sizeof(float), (size_t)ell, cudaMemcpyDefault, h->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->s);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) {
    as_status ds = sync_status(h);
    if (ds != AS_OK) st = ds;
  }
  if (rows_out) *rows_out = (st == AS_OK) ? ell : 0;
  cudaFree(B); cudaFree(lam); cudaFree(V); cudaFree(w); cudaFree(o);
  return st;
}

as_status sketch_get_buffer(as_sketch* h, float* out, int32_t* r_out) {
  if (!h || !out) return AS_EINVAL;
  cudaError_t e = cudaMemcpy2D(out, (size_t)h->d * sizeof(float), h->C, (size_t)h->ldc * sizeof(float),
                               (size_t)h->d * sizeof(float), (size_t)h->n2, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return as_from_cuda(e);
  if (r_out) *r_out = h->r;
  return AS_OK;
}

as_status sketch_get_gram(as_sketch* h, double* out) {
  if (!h || !out) return AS_EINVAL;
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  cudaError_t e = cudaMemcpy(out, h->G, (size_t)h->n2 * h->n2 * sizeof(double), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? AS_OK : as_from_cuda(e);
}

as_status sketch_merge(as_sketch* dst, const as_sketch* src_c) {
  if (!dst || !src_c || dst == src_c) return AS_EINVAL;
  as_sketch* src = const_cast<as_sketch*>(src_c);   // locked and synchronised, not modified
  if (dst->d != src->d) return AS_EINVAL;
  std::unique_lock<std::mutex> l1(dst->mu, std::try_to_lock);
  if (!l1.owns_lock()) return AS_EBUSY;
  std::unique_lock<std::mutex> l2(src->mu, std::try_to_lock);
  if (!l2.owns_lock()) return AS_EBUSY;
  AS_CUDA_TRY(cudaStreamSynchronize(src->s));
  // everything the merge allocates comes first, so a failure leaves dst as it was
  as_status st = ensure_bx(dst);
  if (st == AS_OK) st = ensure_sx(src, dst);
  if (st != AS_OK) return st;
  const int d = dst->d;
  // dst.Bx += src.C^T C + src's snapshot terms + src.Bx: src's whole query Gram
  if (src->r > 0)
    st = gemm_strided<float, float, double>(dst->s, d, d, src->r, src->C, 1, src->ldc, src->C, src->ldc, 1, dst->Bx, d,
                                            1, 1.0, 1.0);
  if (st == AS_OK) st = add_snapshot_terms(src, INT64_MAX, dst->Bx, dst, dst->s);
  if (st == AS_OK && src->Bx) {
    add_f64_kernel<<<256, 256, 0, dst->s>>>(dst->Bx, src->Bx, (size_t)d * d); count_launches(1);
    AS_CUDA_TRY(cudaGetLastError());
  }
  if (st == AS_OK) AS_CUDA_TRY(cudaStreamSynchronize(dst->s));
  return st;
}

as_status sketch_set_theta(as_sketch* h, double theta) {
  if (!h || !(theta >= 0.0)) return AS_EINVAL;
  if (h->mode != AS_FIXED_THETA && h->mode != AS_SITE) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(h->mu, std::try_to_lock);
  if (!lk.owns_lock()) return AS_EBUSY;
  h->theta = theta;
  return AS_OK;
}

as_status sketch_send_snapshots(as_sketch* src, as_sketch* dst, int32_t* sent) {
  if (sent) *sent = 0;
  if (!src || !dst || src == dst || src->d != dst->d) return AS_EINVAL;
  std::unique_lock<std::mutex> l1(dst->mu, std::try_to_lock);
  if (!l1.owns_lock()) return AS_EBUSY;
  std::unique_lock<std::mutex> l2(src->mu, std::try_to_lock);
  if (!l2.owns_lock()) return AS_EBUSY;
  const int32_t n = (int32_t)src->snaps.size();
  if (n == 0) return AS_OK;
  if (src->s != dst->s) AS_CUDA_TRY(cudaStreamSynchronize(src->s));
  as_status st = ensure_bx(dst);
  if (st == AS_OK) st = add_snapshot_terms(src, INT64_MAX, dst->Bx, dst, dst->s);
  if (st != AS_OK) return st;
  // the terms are queued on dst's stream before src's arena can be refilled
  if (src->s != dst->s) AS_CUDA_TRY(cudaStreamSynchronize(dst->s));
  src->snaps.clear();
  src->arena_used = 0;
  src->st.snapshots_sent += n;
  dst->st.snapshots_received += n;
  if (sent) *sent = n;
  return AS_OK;
}

as_status sketch_stats(as_sketch* h, as_stats* out) {
  if (!h || !out) return AS_EINVAL;
  as_status ds = sync_status(h);
  as_stats s = h->st;
  s.rows = h->T;
  s.rows_in_buffer = h->r;
  s.fro2 = h->F;
  s.theta = h->theta;
  s.device_bytes = (int64_t)h->dev_bytes;
  s.device_status = (int32_t)ds;
  s.kernel_launches = as::launches_total();
  *out = s;
  return AS_OK;
}

as_status sketch_trace(as_sketch* h, as_event* out, int64_t cap, int64_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return AS_EINVAL;
  const int64_t n = (int64_t)h->trace.size();
  for (int64_t t = 0; t < std::min(n, cap); ++t) out[t] = h->trace[t];
  *count = n;
  return AS_OK;
}

as_status sketch_profile(as_sketch* h, as_kernel_stat* out, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return AS_EINVAL;
  if (!h->prof) { *count = 0; return AS_OK; }
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  h->prof->resolve();
  int n = 0;
  for (int c = 0; c < PK_COUNT; ++c) {
    if (n < cap) {
      as_kernel_stat& k = out[n];
      std::memset(&k, 0, sizeof(k));
      std::strncpy(k.name, kProfNames[c], sizeof(k.name) - 1);
      k.launches = h->prof->launches[c];
      k.total_ms = h->prof->ms[c];
      k.flops = h->prof->flops[c];
      k.bytes = h->prof->bytes[c];
      k.issued_flops = h->prof->issued[c];
    }
    ++n;
  }
  *count = n;
  return AS_OK;
}

as_status sketch_profile_select(as_sketch* h, uint32_t class_mask) {
  if (!h || !h->prof) return AS_EINVAL;
  AS_CUDA_TRY(cudaStreamSynchronize(h->s));
  h->prof->resolve();
  h->prof->mask = class_mask;
  return AS_OK;
}

as_status sketch_profile_reset(as_sketch* h) {
  if (!h) return AS_EINVAL;
  if (h->prof) {
    AS_CUDA_TRY(cudaStreamSynchronize(h->s));
    h->prof->reset();
  }
  return AS_OK;
}

as_status as_symeig(int32_t n, const double* A, int32_t nev, double* evals, double* vecs) {
  if (n < 1 || nev < 1 || nev > n || !A || !evals || !vecs) return AS_EINVAL;
  const bool big = n > 256;
  double *dA = nullptr, *dl = nullptr, *dX = nullptr, *w = nullptr;
  int* dst = nullptr;
  as_status st = dalloc(&dA, (size_t)n * n);
  if (st == AS_OK) st = dalloc(&dl, (size_t)n);
  if (st == AS_OK) st = dalloc(&dX, (size_t)n * nev);
  if (st == AS_OK) st = dalloc(&w, big ? eig_large_work_doubles(n, nev) : eig_work_doubles(n, nev));
  if (st == AS_OK) st = dalloc(&dst, 1);
  cudaError_t e = cudaSuccess;
  if (st == AS_OK) e = cudaMemset(dst, 0, sizeof(int));
  if (st == AS_OK && e == cudaSuccess) e = cudaMemcpy(dA, A, (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice);
  if (st == AS_OK && e == cudaSuccess)
    st = big ? launch_eig_large(nullptr, n, dA, n, nev, dl, dX, nev, w, nullptr, dst)
             : launch_eig(nullptr, n, dA, n, nev, dl, dX, nev, w);
  if (st == AS_OK && e == cudaSuccess) e = cudaMemcpy(evals, dl, (size_t)nev * sizeof(double), cudaMemcpyDeviceToHost);
  if (st == AS_OK && e == cudaSuccess) e = cudaMemcpy(vecs, dX, (size_t)n * nev * sizeof(double), cudaMemcpyDeviceToHost);
  int ds = 0;
  if (st == AS_OK && e == cudaSuccess) e = cudaMemcpy(&ds, dst, sizeof(int), cudaMemcpyDeviceToHost);
  if (st == AS_OK && e != cudaSuccess) st = as_from_cuda(e);
  if (st == AS_OK && ds != 0) st = (as_status)ds;
  cudaFree(dA); cudaFree(dl); cudaFree(dX); cudaFree(w); cudaFree(dst);
  return st;
}

as_status as_tc_gemm(int32_t M, int32_t N, int32_t K, const float* A, const float* B, int32_t npass, int32_t splits,
                     double* out) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !out || (npass != 1 && npass != 3 && npass != 6) || splits < 1)
    return AS_EINVAL;
  if (!umma_available()) return AS_ENOTSUP;
  const int Kp = (K + 63) / 64 * 64;
  const int bn = umma_bn_for(std::min(N, 256));
  float *dA = nullptr, *dB = nullptr, *dO = nullptr;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr, *a2 = nullptr, *b2 = nullptr;
  int* err = nullptr;
  as_status st = dalloc(&dA, (size_t)M * Kp);
  if (st == AS_OK) st = dalloc(&dB, (size_t)N * Kp);
  if (st == AS_OK) st = dalloc(&ah, (size_t)M * Kp);
  if (st == AS_OK) st = dalloc(&al, (size_t)M * Kp);
  if (st == AS_OK) st = dalloc(&bh, (size_t)N * Kp);
  if (st == AS_OK) st = dalloc(&bl, (size_t)N * Kp);
  if (st == AS_OK) st = dalloc(&a2, (size_t)M * Kp);
  if (st == AS_OK) st = dalloc(&b2, (size_t)N * Kp);
  if (st == AS_OK) st = dalloc(&dO, (size_t)splits * M * N);
  if (st == AS_OK) st = dalloc(&err, 1);
  cudaError_t e = cudaSuccess;
  if (st == AS_OK) {
    e = cudaMemset(dA, 0, (size_t)M * Kp * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(dB, 0, (size_t)N * Kp * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(dO, 0, (size_t)splits * M * N * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy2D(dA, (size_t)Kp * 4, A, (size_t)K * 4, (size_t)K * 4, M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy2D(dB, (size_t)Kp * 4, B, (size_t)K * 4, (size_t)K * 4, N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (st == AS_OK) st = launch_split_bf16(nullptr, dA, Kp, M, Kp, ah, al, Kp, false, a2);
  if (st == AS_OK) st = launch_split_bf16(nullptr, dB, Kp, N, Kp, bh, bl, Kp, false, b2);
  UmmaOperand oa{}, ob{};
  __nv_bfloat16* la[3] = {ah, al, a2};
  __nv_bfloat16* lb[3] = {bh, bl, b2};
  for (int t = 0; t < 3 && st == AS_OK; ++t) {
    st = umma_make_map(&oa.m[t], la[t], M, Kp, Kp, 128);
    if (st == AS_OK) st = umma_make_map(&ob.m[t], lb[t], N, Kp, Kp, bn);
  }
  if (st == AS_OK)
    st = launch_umma_gemm(nullptr, oa, ob, M, N, Kp, bn, npass, splits, 0, dO, N, 1, (long long)M * N, err);
  std::vector<float> h((size_t)splits * M * N);
  int herr = 0;
  if (st == AS_OK) {
    e = cudaMemcpy(h.data(), dO, h.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = as_from_cuda(e);
    if (st == AS_OK && herr) st = (as_status)herr;
  }
  if (st == AS_OK) {
    for (size_t t = 0; t < (size_t)M * N; ++t) {
      double v = 0.0;
      for (int z = 0; z < splits; ++z) v += h[(size_t)z * M * N + t];
      out[t] = v;
    }
  }
  cudaFree(dA); cudaFree(dB); cudaFree(dO); cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(err);
  cudaFree(a2); cudaFree(b2);
  return st;
}

as_status sketch_destroy(as_sketch* h) {
  if (!h) return AS_OK;
  cudaStreamSynchronize(h->s);
  free_all(h);
  delete h;
  return AS_OK;
}

}  // extern "C"

namespace as {
// sketch_update of one of several sketches updated together (the caller runs
// them on separate host threads, each between combined_enter and
// combined_leave, all on the device of combined_begin): FP32 batched iterations share grouped launches.
as_status combined_begin(int dev, void** token) {
  Combiner* c = nullptr;
  as_status st = combiner_for(dev, &c);
  if (st != AS_OK) return st;
  *token = c;
  return AS_OK;
}
void combined_enter(void* token) { static_cast<Combiner*>(token)->enter(); }
void combined_leave(void* token) { static_cast<Combiner*>(token)->leave(); }
as_status sk_update_combined(as_sketch* h, const float* rows, int64_t n, int64_t ld, void* token) {
  return update_rows(h, rows, n, ld, static_cast<Combiner*>(token));
}
}  // namespace as
