// ML-AeroSketch over a sliding window of N rows (Algorithm 6).
//
// Levels j = 0 .. L-1 (L = ceil(log2 R) + 1, so that the level of Fact 1
// exists for every window mass in [N, N R]), each an AeroSketch with the
// fixed threshold theta_j = 2^j eps N and a queue S_j of items (s, t): the
// level's snapshots and the raw rows with ||a||^2 >= theta_j.  For each row
// a_i and each level: pop the queue's front while it holds more than 8/eps
// items or its front is older than the window (t <= i - N); a heavy row is
// queued raw, a light row updates the level's sketch, and a snapshot that
// update takes is queued with t = i.  Every item gets s = (t of the previous
// item) + 1, or 1 on an empty queue.
// Query at time T: the lowest level whose queue is empty or starts at
// s <= max(1, T - N + 1) (the top level if none); B = the level's residual
// C^T C + its queued snapshot terms and raw rows a^T a with t in (T-N, T];
// then the eigen-shrink of Algorithm 5.
//
// A level's sketch computation does not depend on its queue, so a block of
// rows runs each level's sketch over its runs of light rows first, then
// replays the queue row by row on the host and drops the popped snapshots
// from the front of the sketch's own queue.  Each level has its own stream
// and is updated from its own host thread, so the levels' kernels overlap.  A level's sketch numbers its own
// rows (the light rows it received) for its random draws.
#include <algorithm>
#include <cmath>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace {

struct SwItem {
  int64_t s, t;     // interval start and stream time
  int kind;         // 0: snapshot, 1: raw row
  int64_t tint;     // snapshot: the level sketch's own row index
  int slot;         // raw row: slot in the level's ring
};

struct SwLevel {
  as_sketch* h = nullptr;
  cudaStream_t s = nullptr;       // the level's own stream: levels update concurrently
  double theta = 0.0;
  int64_t popped_expired = 0, popped_cap = 0;
  std::deque<SwItem> Q;
  float* ring = nullptr;          // (cap + 2) x d raw rows
  std::vector<int> free_slots;
};

}  // namespace

struct as_sw {
  int d = 0, ell = 0, L = 0, cap = 0;
  int64_t N = 0;
  double eps = 0.0;
  cudaStream_t s = nullptr;
  std::vector<SwLevel> lv;
  int64_t T = 0;
  double* B = nullptr;        // d x d device scratch of the query
  float* rawtmp = nullptr;    // (cap + 2) x d gathered window raw rows
  as_sw_counters st{};
};

extern "C" {

as_status as_sw_destroy(as_sw* w) {
  if (!w) return AS_OK;
  for (SwLevel& l : w->lv) {
    sketch_destroy(l.h);
    if (l.ring) cudaFree(l.ring);
    if (l.s) cudaStreamDestroy(l.s);
  }
  if (w->B) cudaFree(w->B);
  if (w->rawtmp) cudaFree(w->rawtmp);
  delete w;
  return AS_OK;
}

as_status as_sw_create(const as_config* cfg, int64_t N, double R, void* cuda_stream, as_sw** out) {
  if (!cfg || !out || N < 1 || !(R >= 1.0) || std::isinf(R)) return AS_EINVAL;
  *out = nullptr;
  as_sw* w = new (std::nothrow) as_sw();
  if (!w) return AS_ENOMEM;
  w->s = (cudaStream_t)cuda_stream;
  w->N = N;
  w->L = (int)std::ceil(std::log2(R)) + 1;
  as_status st = AS_OK;
  for (int j = 0; j < w->L && st == AS_OK; ++j) {
    as_config c = *cfg;
    c.mode = AS_FIXED_THETA;
    c.stream_id = cfg->stream_id + (uint64_t)j;
    c.theta = 0.0;   // set below once eps is known
    SwLevel l;
    if (cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = AS_EDEVICE;
      break;
    }
    st = sketch_create(&c, l.s, &l.h);
    if (st != AS_OK) {
      cudaStreamDestroy(l.s);
      break;
    }
    if (j == 0) {
      as_stats s0{};
      st = sketch_stats(l.h, &s0);
      w->d = s0.d;
      w->ell = s0.ell;
      w->eps = (cfg->eps > 0.0) ? cfg->eps : 2.0 / s0.ell;
      w->cap = (int)std::floor(8.0 / w->eps);
    }
    l.theta = std::ldexp(1.0, j) * w->eps * (double)N;
    if (st == AS_OK) st = sketch_set_theta(l.h, l.theta);
    w->lv.push_back(l);
  }
  for (SwLevel& l : w->lv) {
    if (st != AS_OK) break;
    if (cudaMalloc((void**)&l.ring, (size_t)(w->cap + 2) * w->d * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      st = AS_ENOMEM;
    }
    for (int k = w->cap + 1; k >= 0; --k) l.free_slots.push_back(k);
  }
  if (st == AS_OK && cudaMalloc((void**)&w->B, (size_t)w->d * w->d * sizeof(double)) != cudaSuccess) st = AS_ENOMEM;
  if (st == AS_OK && cudaMalloc((void**)&w->rawtmp, (size_t)(w->cap + 2) * w->d * sizeof(float)) != cudaSuccess)
    st = AS_ENOMEM;
  if (st != AS_OK) {
    cudaGetLastError();
    as_sw_destroy(w);
    return st;
  }
  w->st.levels = w->L;
  w->st.last_level = -1;
  *out = w;
  return AS_OK;
}

as_status as_sw_update(as_sw* w, const float* rows, int64_t n, int64_t ld) {
  if (!w) return AS_EINVAL;
  if (n == 0) return AS_OK;
  if (!rows || n < 0 || ld < w->d) return AS_EINVAL;
  std::vector<double> nrm((size_t)n);
  as_status st = as::row_norms_f64(rows, n, ld, w->d, w->s, nrm.data());
  if (st != AS_OK) return st;
  for (double v : nrm)
    if (!std::isfinite(v)) return AS_EINVAL;
  // the levels are independent: one host thread per level, each on its own stream
  std::vector<as_status> sts(w->lv.size(), AS_OK);
  auto level_update = [&](SwLevel& l) -> as_status {
    as_status st2 = AS_OK;
    // the level's sketch over its runs of light rows
    const int64_t nl0 = as::sk_rows(l.h);
    const int ns0 = as::sk_snap_count(l.h);
    std::vector<int64_t> light;   // block row of each light row, in order
    for (int64_t t0 = 0; t0 < n;) {
      if (nrm[(size_t)t0] >= l.theta) { ++t0; continue; }
      int64_t t1 = t0;
      while (t1 < n && nrm[(size_t)t1] < l.theta) light.push_back(t1++);
      st2 = sketch_update(l.h, rows + t0 * ld, t1 - t0, ld);
      if (st2 != AS_OK) return st2;
      t0 = t1;
    }
    std::vector<int64_t> snap_at((size_t)n, 0);   // the sketch's row index of a snapshot taken at block row t
    const int ns1 = as::sk_snap_count(l.h);
    for (int k = ns0; k < ns1; ++k) {
      const int64_t tint = as::sk_snap_t(l.h, k);
      snap_at[(size_t)light[(size_t)(tint - nl0 - 1)]] = tint;
    }
    // the queue, row by row
    int drop = 0;
    for (int64_t t = 0; t < n; ++t) {
      const int64_t i = w->T + 1 + t;
      while (!l.Q.empty() && ((int)l.Q.size() > w->cap || l.Q.front().t <= i - w->N)) {
        const SwItem& it = l.Q.front();
        if (it.t <= i - w->N) l.popped_expired += 1; else l.popped_cap += 1;
        if (it.kind == 0) ++drop; else l.free_slots.push_back(it.slot);
        l.Q.pop_front();
      }
      const int64_t s = l.Q.empty() ? 1 : l.Q.back().t + 1;
      if (nrm[(size_t)t] >= l.theta) {
        const int slot = l.free_slots.back();
        l.free_slots.pop_back();
        AS_CUDA_TRY(cudaMemcpyAsync(l.ring + (size_t)slot * w->d, rows + t * ld, (size_t)w->d * sizeof(float),
                                    cudaMemcpyDefault, l.s));
        l.Q.push_back(SwItem{s, i, 1, 0, slot});
      } else if (snap_at[(size_t)t] != 0) {
        l.Q.push_back(SwItem{s, i, 0, snap_at[(size_t)t], -1});
      }
    }
    return as::sk_drop_front(l.h, drop);
  };
  std::vector<std::thread> pool;
  for (size_t j = 0; j < w->lv.size(); ++j) pool.emplace_back([&, j]() { sts[j] = level_update(w->lv[j]); });
  for (std::thread& t : pool) t.join();
  for (as_status s2 : sts)
    if (s2 != AS_OK) return s2;
  w->st.popped_expired = w->st.popped_cap = 0;
  for (const SwLevel& l : w->lv) {
    w->st.popped_expired += l.popped_expired;
    w->st.popped_cap += l.popped_cap;
  }
  w->T += n;
  w->st.rows = w->T;
  return AS_OK;
}

}  // extern "C"

namespace {

int query_level(const as_sw* w) {
  const int64_t lo = std::max<int64_t>(1, w->T - w->N + 1);
  for (int j = 0; j < w->L; ++j) {
    const auto& Q = w->lv[(size_t)j].Q;
    if (Q.empty() || (Q.front().s >= 1 && Q.front().s <= lo)) return j;
  }
  return w->L - 1;
}

// B of the level's window query on the device (w->B).
as_status window_gram(as_sw* w, int j) {
  SwLevel& l = w->lv[(size_t)j];
  const int64_t lb = w->T - w->N;
  int64_t lb_int = INT64_MIN;   // the sketch's index of the last queued snapshot outside the window
  int k = 0;
  for (const SwItem& it : l.Q) {
    if (it.t <= lb) {
      if (it.kind == 0) lb_int = it.tint;
    } else if (it.kind == 1) {
      AS_CUDA_TRY(cudaMemcpyAsync(w->rawtmp + (size_t)k * w->d, l.ring + (size_t)it.slot * w->d,
                                  (size_t)w->d * sizeof(float), cudaMemcpyDeviceToDevice, as::sk_stream(l.h)));
      ++k;
    }
  }
  as_status st = as::sk_window_gram(l.h, lb_int, w->B);
  if (st == AS_OK) st = as::sk_add_rows_gram(l.h, w->rawtmp, k, w->d, w->B);
  return st;
}

}  // namespace

extern "C" {

as_status as_sw_query(as_sw* w, float* out, int64_t ldo, int32_t* rows_out, int32_t* level_out) {
  if (!w || !out || ldo < w->d) return AS_EINVAL;
  const int j = query_level(w);
  as_status st = window_gram(w, j);
  if (st == AS_OK) st = as::sk_eig_shrink(w->lv[(size_t)j].h, w->B, out, ldo);
  if (rows_out) *rows_out = (st == AS_OK) ? w->ell : 0;
  if (level_out) *level_out = j;
  w->st.last_level = j;
  return st;
}

as_status as_sw_query_gram(as_sw* w, double* out, int32_t* level_out) {
  if (!w || !out) return AS_EINVAL;
  const int j = query_level(w);
  as_status st = window_gram(w, j);
  if (st == AS_OK) {
    cudaError_t e = cudaMemcpyAsync(out, w->B, (size_t)w->d * w->d * sizeof(double), cudaMemcpyDeviceToHost,
                                    as::sk_stream(w->lv[(size_t)j].h));
    if (e == cudaSuccess) e = cudaStreamSynchronize(as::sk_stream(w->lv[(size_t)j].h));
    if (e != cudaSuccess) st = as_from_cuda(e);
  }
  if (level_out) *level_out = j;
  w->st.last_level = j;
  return st;
}

as_status as_sw_stats(as_sw* w, as_sw_counters* out) {
  if (!w || !out) return AS_EINVAL;
  w->st.raw_queued = 0;
  w->st.snapshots_queued = 0;
  for (const SwLevel& l : w->lv)
    for (const SwItem& it : l.Q) (it.kind == 1 ? w->st.raw_queued : w->st.snapshots_queued) += 1;
  *out = w->st;
  return AS_OK;
}

as_status as_sw_level(as_sw* w, int32_t j, as_sketch** out) {
  if (!w || !out || j < 0 || j >= w->L) return AS_EINVAL;
  *out = w->lv[(size_t)j].h;
  return AS_OK;
}

}  // extern "C"
