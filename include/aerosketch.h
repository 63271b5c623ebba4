/*
 * aerosketch.h - C ABI of the GB300 AeroSketch update path.
 *
 * AeroSketch (arXiv 2601.02019) keeps a 2l x d residual buffer C, applies the
 * exact Frequent Directions shrink when the buffer is full (Algorithm 4,
 * Section 2.3), gates each update with a power iteration (Algorithm 1 inside
 * Algorithm 4), and moves components whose squared singular value reaches the
 * threshold theta into snapshots (Z, Z^T C'^T C') found by a doubling
 * simultaneous iteration (Algorithm 2 inside Algorithm 4).  A query
 * assembles B = C^T C + the snapshot terms and shrinks it by its l-th
 * eigenvalue (Algorithm 5).  The persistent (ATTP) setting sets
 * theta = eps ||A_t||_F^2 before every update (Algorithm 8).
 *
 * Every function returns an as_status.  Pointers named "host or device" may
 * point to either; the library inspects them.  No function keeps a pointer the
 * caller passed in after it returns.  All work is ordered on the CUDA stream
 * given to sketch_create (NULL = the legacy default stream); functions that
 * return data to the host synchronise that stream.
 *
 * Error behaviour: invalid arguments return AS_EINVAL without side effects;
 * allocation failures return AS_ENOMEM (sketch_update keeps the rows before
 * the one whose step failed; every other call leaves the sketch unchanged);
 * conditions detected on the device (non-finite input, numerical breakdown,
 * a bounded device wait that ran out) are recorded in a sticky status that the
 * next synchronising call returns.
 */
#ifndef AEROSKETCH_H
#define AEROSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct as_sketch as_sketch; /* opaque; owns all of its device memory */

typedef enum {
  AS_OK = 0,
  AS_EINVAL = 1,    /* bad argument or configuration, or non-finite input row */
  AS_ENOMEM = 2,    /* device or host allocation failed */
  AS_EDEVICE = 3,   /* a CUDA call failed */
  AS_ENUMERIC = 4,  /* a factorisation broke down */
  AS_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
  AS_EBUSY = 6,     /* the sketch is in use by another call */
  AS_ENOTSUP = 7    /* valid request that this build does not implement */
} as_status;

/* The stream setting.  The sliding window (Algorithm 6) is a set of
 * AS_FIXED_THETA levels built by as_sw_create; sketch_create returns
 * AS_ENOTSUP for AS_SLIDING. */
typedef enum {
  AS_PERSISTENT = 0,   /* theta = eps ||A_t||_F^2 before every update (Algorithm 8) */
  AS_FIXED_THETA = 1,  /* theta = cfg.theta, changed only by sketch_set_theta (Algorithm 3) */
  AS_SLIDING = 2,      /* Algorithm 6: use as_sw_create (sketch_create: AS_ENOTSUP) */
  AS_SITE = 3,         /* Algorithm 10, a site: as AS_FIXED_THETA (cfg.theta may be +inf); its
                          snapshots are moved to a coordinator by sketch_send_snapshots */
  AS_COORDINATOR = 4   /* Algorithm 10, the coordinator: no rows (sketch_update returns
                          AS_EINVAL); accumulates received snapshot terms; its query is
                          the eigen-shrink of Algorithm 5 on that sum */
} as_mode;

/* Arithmetic of the products.  In every form the orthonormalisations and the
 * Rayleigh-Ritz steps run in FP64; the eigensolver of the FD shrink (and of
 * queries with d > 256) runs in double-float arithmetic (df64: pairs of FP32
 * values, about 48 significant bits; its O(n) scalars and inverse iteration
 * in FP64), the smaller eigendecompositions in FP64.  Every branch of
 * Algorithm 4 is decided on FP64 values (values inside a 1e-4 relative band
 * of a threshold are recomputed in FP64).
 *   AS_FP32_PLAIN  SIMT FP32 products, FP32 partial sums combined in FP64.
 *   AS_BF16        d-side products (Gram rows, FD rebuild) on the tcgen05
 *                  tensor cores with BF16 operands and FP32 accumulation;
 *                  batched G-space products (the decision iterations) in
 *                  two-level split-BF16 on tcgen05 for blocks of 256 or more
 *                  padded rows, in FP32 SIMT below that.
 *   AS_BF16X3      as AS_BF16 with the d-side products in two-level split-BF16
 *                  (x = hi + lo; hi*hi + hi*lo + lo*hi: ~16-bit operands).
 *   AS_BF16X6      as AS_BF16 with the d-side products in three-level
 *                  split-BF16 (x = hi + mid + lo, the six products above
 *                  2^-24: operands as exact as FP32). */
typedef enum {
  AS_FP32_PLAIN = 0,
  AS_BF16 = 1,
  AS_BF16X3 = 2,
  AS_BF16X6 = 3
} as_precision;

/* Flags. */
#define AS_TRACE_DECISIONS 0x1u /* record every gate / doubling decision (sketch_trace) */
#define AS_PROFILE 0x2u         /* time each kernel class with CUDA events (sketch_profile) */
#define AS_QUERY_DENSE 0x4u     /* sketch_query always takes the dense d x d route (see sketch_query) */

typedef struct {
  int32_t d;          /* row dimension, >= 2 */
  int32_t ell;        /* sketch size l, 1 <= l <= d/2 (Section 2.3); 0 => ceil(2/eps) */
  double eps;         /* error parameter; 0 => 2/l (Algorithm 3) */
  int32_t mode;       /* as_mode */
  int32_t prec;       /* as_precision */
  double theta;       /* dump threshold for AS_FIXED_THETA (may be +inf) */
  double eps_si;      /* simultaneous-iteration accuracy; 0 => 0.4 (Algorithm 4) */
  int32_t k_pi;       /* power iterations; 0 => ceil(log2 d) + 1 (Corollary 1) */
  int32_t q_si;       /* simultaneous-iteration products; 0 => ceil(ln d / eps_si) */
  uint64_t seed;      /* Philox key word 0 for the method's random draws */
  uint64_t stream_id; /* Philox key word 1 */
  uint32_t flags;     /* AS_TRACE_DECISIONS | AS_PROFILE */
  uint32_t reserved;
  double delta;       /* probability amplification (Algorithm 7): 0 = off, else the
                         failure probability delta in (0, 1): at every doubling step
                         r = ceil(log_100(2/delta)) simultaneous iterations with
                         eps_SI = 0.2 are run and the one whose residual has the smallest
                         maximum of s = ceil(2 log_3(2/delta)) power-iteration estimates
                         is kept; SI h draws its test matrix at Philox sub-index
                         j + 64 (h-1), estimate g of SI h its start vector at 64 h + g.
                         Every row whose gate passes takes the FP64 single-row path.
                         AS_EINVAL unless r <= 15 and s <= 63 (delta >~ 2e-15). */
} as_config;

typedef struct {
  int64_t rows;            /* rows ingested (the current time T) */
  int32_t ell, d;
  int32_t rows_in_buffer;  /* r: filled rows of C */
  int32_t reserved0;
  double fro2;             /* ||A_T||_F^2 (FP64) */
  double theta;            /* threshold in force after the last update */
  int64_t shrinks;         /* FD shrinks (Algorithm 4) */
  int64_t gates;           /* rows whose power-iteration gate passed */
  int64_t dumps;           /* snapshots taken */
  int64_t snapshot_rank;   /* sum of xi over the snapshot queue */
  int64_t si_runs;         /* simultaneous iterations run */
  int64_t device_bytes;    /* device memory owned by the sketch */
  int32_t device_status;   /* sticky as_status recorded on the device */
  int32_t reserved1;
  int64_t kernel_launches; /* kernels this library launched, all sketches, since load */
  int64_t snapshots_sent;      /* snapshots moved out by sketch_send_snapshots */
  int64_t snapshots_received;  /* snapshots accumulated from other sketches */
  int64_t grouped_batches;     /* blocks whose batched iterations ran in a launch shared with other sketches */
} as_stats;

/* Per kernel class timing (AS_PROFILE): CUDA-event time on the sketch's
 * stream, launch count, and the algorithmic work of those launches. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double flops;     /* algorithmic floating-point operations, summed over launches.  For the
                       batched iterations ("batch_tc", "batch_persist"): the power iterations
                       of the rows whose gate they decided and the k = 2 simultaneous
                       iterations of the gated rows that used them, 2 m_t^2 per product */
  double bytes;     /* algorithmic DRAM bytes, summed over launches */
  double issued_flops;  /* floating-point operations the launches issued (for the batched
                           iterations: every row of every block, including the rows after a
                           block's first state-changing row, which are fed again) */
} as_kernel_stat;

/* One decision record (AS_TRACE_DECISIONS): a row whose gate passed. */
typedef struct {
  int64_t i;        /* timestamp of the row (1-based) */
  double sig2_pi;   /* power-iteration estimate sigma_hat_1^2 (Algorithm 1) */
  double theta;     /* threshold in force */
  int32_t j_stop;   /* doubling step that broke the loop, 0 if none */
  int32_t xi;       /* components dumped, xi (Algorithm 4) */
  double ritz_k;    /* sigma_hat_k^2 at the stopping step (or the last one) */
  double ritz_1;    /* sigma_hat_1^2 at that step */
  uint64_t amp_choice; /* with probability amplification: the simultaneous
                          iteration kept at doubling step j (1-based, 0 = none)
                          in bits 4(j-1) .. 4(j-1)+3 */
} as_event;

/* Create a sketch (Algorithm 3, and Algorithm 8's Initialize for
 * AS_PERSISTENT).  `cuda_stream` is a cudaStream_t or NULL.  Allocates C
 * (2l x d, FP32), G = C C^T (2l x 2l, FP64) and work space on the current
 * device.  Returns AS_EINVAL for d < 2, l < 1, 2l > d, eps <= 0 or an unknown
 * mode; AS_ENOTSUP for a mode or precision this build does not implement. */
as_status sketch_create(const as_config* cfg, void* cuda_stream, as_sketch** out);

/* Feed n rows (Algorithm 4 for each row, preceded by Algorithm 8's threshold
 * update in AS_PERSISTENT mode).  `rows` is host or device memory holding n
 * rows of d FP32 values, row t at rows + t*ld (ld >= d).  n = 0 is a no-op.
 * The call returns once the rows are consumed; `rows` may then be reused.
 * Returns AS_EINVAL (and ingests nothing from that row on) if a row holds a
 * non-finite value. */
as_status sketch_update(as_sketch* h, const float* rows, int64_t n, int64_t ld);

/* Algorithm 8's Query(t) = Algorithm 5 with lb = 0, ub = t: writes the
 * l x d sketch B_hat, row-major with leading dimension ldo >= d, to `out`
 * (host or device), and the number of rows written (l) to *rows_out.
 * t = -1 or t = T (rows fed so far) is the current time: B = C_T^T C_T plus
 * every snapshot term.  0 <= t < T is a historical time: the residual C_t is
 * not stored, and B is the sum of the snapshot terms taken at rows <= t (the
 * B_t of the ATTP error analysis).  Other t: AS_EINVAL.  Synchronises.
 * Route: B = F^T H F with F the r_F stacked factor rows [C; Z_j^T; Y_j] and a
 * small block-diagonal H.  When r_F <= 3d/4 (and the sketch holds no merged
 * terms) the eigenpairs come from two r_F x r_F eigenproblems (the Gram of F
 * and the core matrix on its row space); otherwise, or with AS_QUERY_DENSE,
 * from the d x d matrix B.  Both routes give the same B_hat up to rounding and
 * the signs of its rows. */
as_status sketch_query(as_sketch* h, int64_t t, float* out, int64_t ldo, int32_t* rows_out);

/* The matrix B of Algorithm 5 (before its eigendecomposition) for the time t of sketch_query
 * (before its eigendecomposition): d x d FP64, row-major, to host memory
 * `out`.  Synchronises. */
as_status sketch_query_gram(as_sketch* h, int64_t t, double* out);

/* Copy the residual buffer C (2l x d FP32, row-major, leading dimension d)
 * and the row count r to host memory.  Synchronises. */
as_status sketch_get_buffer(as_sketch* h, float* out, int32_t* r_out);

/* Copy the maintained Gram matrix G = C C^T of the buffer (2l x 2l FP64,
 * row-major) to host memory.  G feeds the power iteration, the simultaneous
 * iteration and the FD shrink's eigendecomposition; it should equal the Gram
 * of the rows sketch_get_buffer returns.  Synchronises. */
as_status sketch_get_gram(as_sketch* h, double* out);

/* Merge src into dst by decomposability (Appendix E: the covariance of a
 * union of streams is the sum of the parts', and the errors add): dst
 * accumulates src's whole query Gram, C^T C plus every snapshot term plus
 * what src itself absorbed, in a d x d FP64 accumulator that dst's
 * current-time query adds to its own B.  src is not modified.  Requires equal
 * d (AS_EINVAL otherwise; also for dst == src).  Synchronises both streams. */
as_status sketch_merge(as_sketch* dst, const as_sketch* src);

/* Set the dump threshold theta (>= 0, +inf allowed) of an AS_FIXED_THETA or
 * AS_SITE sketch; it applies from the next row on.  Algorithm 10: a site sets
 * theta when it receives the coordinator's broadcast.  Other modes or a
 * negative or NaN theta: AS_EINVAL. */
as_status sketch_set_theta(as_sketch* h, double theta);

/* Algorithm 10, site side: send every snapshot in src's queue to dst (the
 * coordinator, or any sketch of the same d) and delete them from src's queue.
 * dst adds each term Z Y + Y^T Z^T - Z (Y Z) Z^T to its d x d FP64
 * accumulator, in time order, on dst's stream.  *sent (may be NULL) receives
 * the number of snapshots moved.  Requires equal d. */
as_status sketch_send_snapshots(as_sketch* src, as_sketch* dst, int32_t* sent);

/* ---- P5: distributed sites and coordinator (Algorithm 10) --------------
 * m AS_SITE sketches (each on a stream of its own, updated from the library's
 * worker threads so that their kernels overlap) and one AS_COORDINATOR
 * sketch on cuda_stream, driven in synchronous rounds.  Per row of site j: F_j += ||a||^2; when F_j >=
 * (eps/m) F_hat (the last broadcast value) the site messages F_j and resets
 * it; the row updates site j; site j's snapshots are then sent to the
 * coordinator.  At the end of a round the coordinator adds the messages in
 * site order and, at every m-th message, broadcasts F_hat: each site's
 * threshold becomes (eps/m) F_hat (the per-site error of the analysis; the
 * algorithm text prints eps F_hat).  Sites start with theta = +inf
 * (Algorithm 10 leaves it open): nothing is sent before the first broadcast.
 * Site j uses Philox stream_id = site_cfg->stream_id + j. */
typedef struct as_p5 as_p5;

typedef struct {
  int64_t rounds, messages, broadcasts, snapshots_sent;
  double f_hat;    /* the coordinator's F_hat */
  double f_site;   /* F_hat as the sites know it (last broadcast) */
} as_p5_counters;

/* site_cfg: the sites' configuration (mode and theta are overridden).  m >= 1.
 * AS_EINVAL on bad arguments; errors of sketch_create are passed through. */
as_status as_p5_create(const as_config* site_cfg, int32_t m, void* cuda_stream, as_p5** out);
/* One synchronous round: rows[j] (host or device, n[j] rows of d FP32 values,
 * row stride ld[j] >= d) are site j's rows; n[j] = 0 is allowed. */
as_status as_p5_round(as_p5* p, const float* const* rows, const int64_t* n, const int64_t* ld);
/* The coordinator's Query (the eigen-shrink of Algorithm 5 on B): l x d, as sketch_query. */
as_status as_p5_query(as_p5* p, float* out, int64_t ldo, int32_t* rows_out);
/* The coordinator's B (d x d FP64, host memory). */
as_status as_p5_query_gram(as_p5* p, double* out);
as_status as_p5_stats(as_p5* p, as_p5_counters* out);
/* Borrowed handles (owned by p): site j, the coordinator. */
as_status as_p5_site(as_p5* p, int32_t j, as_sketch** out);
as_status as_p5_coordinator(as_p5* p, as_sketch** out);
/* Destroy p, its sites and its coordinator.  NULL is a no-op. */
as_status as_p5_destroy(as_p5* p);

/* ---- Sliding window: ML-AeroSketch (Algorithm 6) ------------------------
 * The sketch of the last N rows.  L = ceil(log2 R) + 1 levels (R: an upper
 * bound of the rows' squared norms, >= 1), level j an AS_FIXED_THETA sketch
 * with theta_j = 2^j eps N (Philox stream_id = cfg->stream_id + j) and a
 * queue of its snapshots and of the raw rows with ||a||^2 >= theta_j, at
 * most 8/eps items, items older than the window dropped.  Each queued item
 * carries s = (t of the previous item) + 1, or 1 on an empty queue (the
 * snapshot rule of Algorithm 4, read for raw rows too).  The query answers
 * from the lowest level whose queue is empty or starts at s <= max(1,
 * T - N + 1) (the top level if none), with B = its residual C^T C + its
 * queued snapshot terms and raw rows a^T a in (T-N, T], then the eigen-shrink
 * of Algorithm 5.  A level's sketch numbers its own rows for its random draws. */
typedef struct as_sw as_sw;

typedef struct {
  int64_t rows;               /* T: rows fed */
  int32_t levels, last_level; /* L; the level of the last query (-1 before any) */
  int64_t raw_queued, snapshots_queued;   /* items in all queues now */
  int64_t popped_expired, popped_cap;     /* items dropped by age, by the 8/eps cap */
} as_sw_counters;

/* cfg: d, ell or eps, prec, seed, stream_id of the levels (mode and theta
 * are overridden).  N >= 1; R >= 1 and finite.  AS_EINVAL on bad arguments. */
as_status as_sw_create(const as_config* cfg, int64_t N, double R, void* cuda_stream, as_sw** out);
/* Feed n rows (host or device, row stride ld >= d); a non-finite row: AS_EINVAL,
 * nothing of the call ingested. */
as_status as_sw_update(as_sw* w, const float* rows, int64_t n, int64_t ld);
/* The l x d sketch of the window (T-N, T] (as sketch_query); *level_out (may be
 * NULL) receives the level that answered.  Synchronises. */
as_status as_sw_query(as_sw* w, float* out, int64_t ldo, int32_t* rows_out, int32_t* level_out);
/* The window's B (d x d FP64, host memory) before its eigendecomposition. */
as_status as_sw_query_gram(as_sw* w, double* out, int32_t* level_out);
as_status as_sw_stats(as_sw* w, as_sw_counters* out);
/* Borrowed handle of level j's sketch (owned by w). */
as_status as_sw_level(as_sw* w, int32_t j, as_sketch** out);
/* Destroy w and its levels.  NULL is a no-op. */
as_status as_sw_destroy(as_sw* w);

/* ---- Footprint, grouped updates and the serving runtime ------------------
 *
 * Many independent sketches (sessions, levels, sites) progress at once: each
 * on a stream of its own, driven by host worker threads, so that their
 * kernels overlap on the GPU; or with their batched iterations sharing
 * cooperative launches through a launch combiner (sketch_update_grouped).  A sketch's kernels and launch shapes depend only
 * on its own configuration and rows, so its results are bitwise the same
 * alone and in any mix. */

/* Device bytes a sketch of configuration cfg holds once sketch_reserve(h,
 * snapshot_rank) has run: the state sketch_create allocates, the buffers that
 * otherwise grow on demand at their maxima, and a snapshot store for snapshots
 * of total rank snapshot_rank (2 d floats per unit of rank: Z and Y).  With
 * ATTP (Algorithm 8) the total snapshot rank after T rows is at most
 * (2/eps) ln(2 ||A_T||_F^2 / (eps ||A_1||_F^2)) (the space analysis of Algorithm 8).
 * Host arithmetic only: no allocation, no device call (AS_ENOTSUP for the tensor
 * forms without a device).  AS_EINVAL for a bad configuration. */
as_status sketch_footprint(const as_config* cfg, int64_t snapshot_rank, int64_t* bytes);

/* Allocate now what sketch_footprint counts: the on-demand buffers at their
 * maxima and room for snapshot_rank more units of snapshot rank.  After it, the
 * sketch's device_bytes equals the footprint.  A larger rank later still
 * grows the store. */
as_status sketch_reserve(as_sketch* h, int64_t snapshot_rank);

/* Update `count` sketches, sketch k with rows[k] (n[k] rows, stride ld[k], host
 * or device), each progressing independently on the library's worker
 * threads (at most 16), each on the stream it was created with (sketches
 * created on streams of their own overlap their kernels on the GPU).  Entries naming the same sketch run in list order.
 * Blocks until all are done; returns AS_OK or the status of the first failing
 * entry in list order (the other entries still run).  The caller keeps the
 * rows valid until the call returns. */
as_status sketch_update_many(as_sketch* const* hs, const float* const* rows, const int64_t* n, const int64_t* ld,
                             int32_t count);

/* The same update with the sketches' batched iterations in shared launches:
 * every sketch progresses on a worker thread of its own, as in
 * sketch_update_many, but a block whose FP32 batched iterations (the power
 * iteration and first simultaneous-iteration step of every row) are ready is
 * handed to the device's launch combiner, which runs the pending blocks of all
 * sketches in one cooperative launch (as_stats.grouped_batches counts them) as
 * soon as every sketch of the call has a block pending, or 40 us after the
 * first one arrived.  No sketch waits for another's decisions.  Each sketch's
 * results are bitwise those of sketch_update on its rows.  Arguments, ordering
 * and errors as sketch_update_many; all sketches must live on one device
 * (AS_EINVAL otherwise). */
as_status sketch_update_grouped(as_sketch* const* hs, const float* const* rows, const int64_t* n, const int64_t* ld,
                                int32_t count);

/* The serving runtime: sessions (one persistent-mode sketch each, on a stream
 * of its own) admitted against an HBM budget by their footprint; requests
 * (a batch of rows for one session) queued and run by worker threads with
 * continuous batching: a free worker takes the session whose oldest pending
 * request is the oldest, so requests of different sessions run concurrently and
 * each session's requests run in submission order. */
typedef struct as_server as_server;

typedef struct {
  int64_t hbm_budget;   /* bytes the sessions may hold; 0 = 90% of the device's free memory at create */
  int32_t workers;      /* worker threads, 1..64 (0 = 16) */
  int32_t reserved;
} as_server_config;

typedef struct {
  int64_t sessions_open;
  int64_t sessions_refused;   /* opens refused for the budget (AS_EBUSY) */
  int64_t footprint_bytes;    /* the open sessions' footprints */
  int64_t requests_done;      /* completed requests (since the last reset) */
  int64_t requests_failed;
  int64_t rows_done;
  double p50_ms, p99_ms, max_ms, mean_ms;   /* latency: completion - submission, completed requests */
  double span_s;              /* first submission to last completion since the last reset */
} as_server_counters;

as_status as_server_create(const as_server_config* cfg, as_server** out);
/* Open a persistent-mode session (cfg->mode must be AS_PERSISTENT).  Its
 * footprint is sketch_footprint(cfg, rank) with rank = the snapshot bound
 * above for mass_ratio = ||A_T||_F^2 / ||A_1||_F^2 >= 1 (the caller's bound on
 * the session's growth).  AS_EBUSY if the open sessions' footprints plus this
 * one exceed the budget (nothing allocated); *session receives an id > 0. */
as_status as_server_open(as_server* sv, const as_config* cfg, double mass_ratio, int64_t* session);
/* Queue n rows (host or device, stride ld) for a session; *ticket (may be
 * NULL) receives the request's id.  The caller keeps the rows valid until the
 * request completes (as_server_wait or as_server_drain). */
as_status as_server_submit(as_server* sv, int64_t session, const float* rows, int64_t n, int64_t ld,
                           int64_t* ticket);
/* Wait for one request; returns its status, *latency_ms (may be NULL) its
 * completion - submission time.  A ticket can be waited on once. */
as_status as_server_wait(as_server* sv, int64_t ticket, double* latency_ms);
/* Wait until no request is pending or running; returns the first failure
 * status among the requests completed since the last drain, else AS_OK. */
as_status as_server_drain(as_server* sv);
/* Borrowed handle of a session's sketch (owned by the server) for queries and
 * stats; use it only while the session has no pending request. */
as_status as_server_session(as_server* sv, int64_t session, as_sketch** out);
/* Close a session with no pending request (AS_EBUSY otherwise), freeing its
 * footprint. */
as_status as_server_close(as_server* sv, int64_t session);
as_status as_server_stats(as_server* sv, as_server_counters* out);
/* Clear the latency record, the request counters and the span. */
as_status as_server_reset_stats(as_server* sv);
/* Stop the workers (after the running requests), close every session. */
as_status as_server_destroy(as_server* sv);

/* Self-test of the library's bounded device waits: runs one of them on
 * something that nothing completes (kind 0: a release flag, 1: a grid
 * barrier, 2: an mbarrier phase) with a limit of limit_ms (1..2000) in one
 * small kernel on cuda_stream.  Returns AS_ETIMEOUT when the wait gave up as
 * designed (the device context stays usable), AS_OK if it did not, AS_EINVAL
 * for bad arguments.  Synchronises.  Production waits use a 2 s limit. */
as_status as_wait_selftest(int32_t kind, int32_t limit_ms, void* cuda_stream);

/* Counters and the sticky device status.  Synchronises. */
as_status sketch_stats(as_sketch* h, as_stats* out);

/* Decision records (AS_TRACE_DECISIONS).  Copies up to `cap` records, oldest
 * first, to host memory `out` and writes the total count to *count. */
as_status sketch_trace(as_sketch* h, as_event* out, int64_t cap, int64_t* count);

/* Kernel-class timings collected since the last reset (AS_PROFILE).
 * Synchronises; copies up to `cap` records to host memory `out` and writes the
 * number of classes to *count.  Without AS_PROFILE, *count = 0. */
as_status sketch_profile(as_sketch* h, as_kernel_stat* out, int32_t cap, int32_t* count);

/* Clear the kernel-class timings. */
as_status sketch_profile_reset(as_sketch* h);

/* Restrict the AS_PROFILE timing to the kernel classes whose bits are set in
 * class_mask: bit c stands for entry c of sketch_profile's list (a fixed
 * order).  The other classes are no longer bracketed with CUDA events, which
 * takes their event records (host calls on every block) off the update path;
 * their counters stop growing.  All classes are timed by default.  A library
 * service with no counterpart in the paper.  AS_EINVAL without AS_PROFILE. */
as_status sketch_profile_select(as_sketch* h, uint32_t class_mask);

/* Symmetric eigendecomposition on the current device, FP64 in and out: the
 * core factorisation that the FD shrink (Algorithm 4, through the Gram matrix
 * of the buffer) and the query (Algorithm 5) use.  n <= 256: one thread block
 * in FP64; n > 256: the GPU-wide solver in df64 (about 48 significant bits).
 * A is n x n, row-major, host memory (only its values are read; it is not
 * modified).
 * Writes the nev largest eigenvalues in descending order to evals (host) and
 * the matching unit eigenvectors as the columns of vecs (host, n x nev,
 * row-major).  1 <= nev <= n.  Synchronous. */
as_status as_symeig(int32_t n, const double* A, int32_t nev, double* evals, double* vecs);

/* The tensor-core product that the BF16 forms use for their d-side and
 * G-space contractions: out = A B^T with A (M x K) and B (N x K) FP32,
 * row-major, host memory, computed by the tcgen05 kernel with BF16 operands
 * and FP32 accumulation: npass = 1 rounds the operands to BF16 once, npass =
 * 3 uses the two-level split-BF16 form (hi*hi + hi*lo + lo*hi), npass = 6 the
 * three-level one (all products of levels i + j <= 2).  `splits` > 1 splits K
 * across thread blocks (partials summed in FP64 here).  out: M x N row-major
 * host memory.  Synchronous.  AS_ENOTSUP if the driver lacks tensor-map support. */
as_status as_tc_gemm(int32_t M, int32_t N, int32_t K, const float* A, const float* B, int32_t npass, int32_t splits,
                     double* out);

/* as_symeig without any allocation, for callers that cannot allocate device
 * memory: allocator callbacks, and real-time serving paths that forbid
 * allocation after start-up.  The paper has no counterpart: this is a library
 * service.  A (n x n, row-major, device memory, not modified), evals (nev,
 * device) and vecs (n x nev row-major, device) are the caller's; the scratch
 * space is a fixed device array of 788,992 bytes inside the library, reserved
 * on every GPU that loads it until the process exits.  n must be <= 128
 * (AS_EINVAL otherwise).  Work is ordered on cuda_stream (NULL = legacy default
 * stream) and the call returns without synchronising.  All calls share the
 * scratch array and it keeps the last call's contents (every value the solver
 * reads is written earlier in the same call): calls that overlap on the GPU
 * race.  The first call on a device, and the first after that device's
 * context was destroyed and made again (cudaDeviceReset), looks up the array's
 * address (cudaGetSymbolAddress, no allocation); make that first call on each
 * device before any stream capture begins.  AS_ENOTSUP if the
 * driver entry point for the current context cannot be found. */
as_status as_symeig_noalloc(int32_t n, const double* A, int32_t nev, double* evals, double* vecs, void* cuda_stream);

/* Free every resource of the sketch.  NULL is a no-op. */
as_status sketch_destroy(as_sketch* h);

/* Test hook for the allocation-failure paths (a library service; the paper
 * has no counterpart): after `after` >= 0 more successful device allocations
 * made by sketches of this library (any thread), the next one fails as if the
 * device were out of memory, and the hook turns itself off; after = -1 turns
 * it off at once.  AS_EINVAL for after < -1.  A failing sketch_create frees
 * what it allocated; a failing query, merge or sketch_reserve leaves the
 * sketch as it was; a failing sketch_update keeps the rows before the one
 * whose step needed the allocation. */
as_status as_inject_alloc_failure(int32_t after);

/* Static string naming a status. */
const char* as_status_str(as_status s);

/* The last CUDA call of this library that failed on the calling thread, as
 * "<cudaError name> (<source file>:<line>)"; "" if none.  Library service
 * (the paper has no counterpart).  The string is owned by the library and
 * valid until the thread's next failing call. */
const char* as_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AEROSKETCH_H */
