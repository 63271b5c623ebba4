// Grouped updates of many sketches and the serving runtime: host C++ over the
// sketch calls.  Independent sketches (the serving sessions, and in general any
// set of streams to be sketched at once) each own a CUDA stream; host worker
// threads drive them so that their kernels overlap on the GPU.  Nothing here
// touches a sketch's arithmetic: a session's results are those of
// sketch_update on its own rows, bitwise, whatever else runs beside it.
//
// Admission (the space analysis of Algorithm 8): with ATTP the snapshots a
// sketch stores after T rows have total rank at most
// (2/eps) ln(2 ||A_T||_F^2 / (eps ||A_1||_F^2)), so a session's device memory
// is bounded by its fixed state plus 2 d floats per unit of that rank; the
// server admits a session only while the sum of these bounds fits its budget,
// and allocates the bound up front (sketch_reserve) so that a running session
// never grows past what was admitted.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// A fixed set of host threads running queued tasks (sketch_update_many).
class Pool {
 public:
  explicit Pool(int n) {
    for (int t = 0; t < n; ++t) th_.emplace_back([this]() { loop(); });
  }
  void run(std::function<void()> f) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      q_.push_back(std::move(f));
    }
    cv_.notify_one();
  }

 private:
  void loop() {
    for (;;) {
      std::function<void()> f;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&]() { return !q_.empty(); });
        f = std::move(q_.front());
        q_.pop_front();
      }
      f();
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<std::function<void()>> q_;
  std::vector<std::thread> th_;
};

// The pool lives for the whole process (its idle threads end with it).
Pool& pool() {
  static Pool* p = new Pool(16);
  return *p;
}

struct Latch {
  std::mutex mu;
  std::condition_variable cv;
  size_t left;
  explicit Latch(size_t n) : left(n) {}
  void done() {
    std::lock_guard<std::mutex> lk(mu);
    if (--left == 0) cv.notify_all();
  }
  void wait() {
    std::unique_lock<std::mutex> lk(mu);
    cv.wait(lk, [&]() { return left == 0; });
  }
};

// Total snapshot rank bound of the ATTP space analysis, (2/eps) ln(2 R / eps)
// for the mass ratio R = ||A_T||^2 / ||A_1||^2, rounded up.
int64_t attp_rank_bound(double eps, double ratio) {
  const double v = (2.0 / eps) * std::log(2.0 * ratio / eps);
  return (int64_t)std::ceil(std::max(v, 0.0));
}

double percentile(std::vector<double> v, double p) {   // nearest rank
  if (v.empty()) return 0.0;
  size_t k = (size_t)std::ceil(p * (double)v.size());
  k = std::min(std::max<size_t>(k, 1), v.size()) - 1;
  std::nth_element(v.begin(), v.begin() + (long)k, v.end());
  return v[k];
}

}  // namespace

namespace as {

void run_parallel(int n, const std::function<void(int)>& f) {
  if (n <= 0) return;
  if (n == 1) {
    f(0);
    return;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  Latch latch((size_t)n);
  for (int i = 0; i < n; ++i)
    pool().run([&, i]() {
      cudaSetDevice(dev);
      f(i);
      latch.done();
    });
  latch.wait();
}

}  // namespace as

struct as_server {
  struct Session {
    as_sketch* h = nullptr;
    cudaStream_t s = nullptr;
    int64_t footprint = 0;
    std::deque<int64_t> pending;   // tickets, in submission order
    bool running = false;
  };
  struct Request {
    int64_t session = 0;
    const float* rows = nullptr;
    int64_t n = 0, ld = 0;
    Clock::time_point t0;
    bool done = false;
    as_status st = AS_OK;
    double lat_ms = 0.0;
  };
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int64_t, Session> sessions;
  std::unordered_map<int64_t, Request> reqs;
  std::set<std::pair<int64_t, int64_t>> ready;   // (oldest pending ticket, session), nothing running
  std::vector<std::thread> workers;
  bool stop = false;
  int dev = 0;
  int64_t next_session = 1, next_ticket = 1;
  int64_t budget = 0, used = 0;
  int64_t outstanding = 0;        // submitted, not completed
  as_status first_fail = AS_OK;   // since the last drain
  // counters since the last reset
  std::vector<double> lat;
  int64_t done_n = 0, failed_n = 0, rows_n = 0, refused = 0;
  bool have_t0 = false;
  Clock::time_point first_submit, last_done;

  void work() {
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv_work.wait(lk, [&]() { return stop || !ready.empty(); });
      if (ready.empty()) return;   // stop, and nothing left to start
      const int64_t sid = ready.begin()->second;
      ready.erase(ready.begin());
      Session& S = sessions[sid];
      const int64_t t = S.pending.front();
      S.pending.pop_front();
      S.running = true;
      const Request r = reqs[t];
      lk.unlock();
      const as_status st = sketch_update(S.h, r.rows, r.n, r.ld);
      const Clock::time_point t1 = Clock::now();
      lk.lock();
      Request& R = reqs[t];
      R.done = true;
      R.st = st;
      R.lat_ms = std::chrono::duration<double, std::milli>(t1 - r.t0).count();
      lat.push_back(R.lat_ms);
      ++done_n;
      if (st == AS_OK) rows_n += r.n;
      else {
        ++failed_n;
        if (first_fail == AS_OK) first_fail = st;
      }
      last_done = t1;
      S.running = false;
      if (!S.pending.empty()) {
        ready.emplace(S.pending.front(), sid);
        cv_work.notify_one();
      }
      --outstanding;
      cv_done.notify_all();
    }
  }
};

extern "C" {

as_status sketch_update_many(as_sketch* const* hs, const float* const* rows, const int64_t* n, const int64_t* ld,
                             int32_t count) {
  if (count < 0) return AS_EINVAL;
  if (count == 0) return AS_OK;
  if (!hs || !rows || !n || !ld) return AS_EINVAL;
  for (int32_t k = 0; k < count; ++k)
    if (!hs[k]) return AS_EINVAL;
  if (count == 1) return sketch_update(hs[0], rows[0], n[0], ld[0]);
  // entries grouped by sketch, each group in list order, one worker per sketch
  std::vector<std::vector<int32_t>> groups;
  std::unordered_map<const as_sketch*, size_t> gi;
  for (int32_t k = 0; k < count; ++k) {
    auto it = gi.find(hs[k]);
    if (it == gi.end()) {
      gi.emplace(hs[k], groups.size());
      groups.push_back({k});
    } else {
      groups[it->second].push_back(k);
    }
  }
  std::vector<as_status> st((size_t)count, AS_OK);
  as::run_parallel((int)groups.size(), [&](int g) {
    for (int32_t k : groups[(size_t)g]) st[(size_t)k] = sketch_update(hs[k], rows[k], n[k], ld[k]);
  });
  for (as_status e : st)
    if (e != AS_OK) return e;
  return AS_OK;
}

as_status sketch_update_grouped(as_sketch* const* hs, const float* const* rows, const int64_t* n, const int64_t* ld,
                                int32_t count) {
  if (count < 0) return AS_EINVAL;
  if (count == 0) return AS_OK;
  if (!hs || !rows || !n || !ld) return AS_EINVAL;
  for (int32_t k = 0; k < count; ++k)
    if (!hs[k]) return AS_EINVAL;
  // every sketch on a host thread of its own, its FP32 batched iterations
  // grouped with whichever other sketches have a block ready (the device's
  // launch combiner)
  const int dev = as::sk_device(hs[0]);
  for (int32_t k = 1; k < count; ++k)
    if (as::sk_device(hs[k]) != dev) return AS_EINVAL;
  void* comb = nullptr;
  {
    const as_status cs = as::combined_begin(dev, &comb);
    if (cs != AS_OK) return cs;
  }
  std::vector<std::vector<int32_t>> groups;
  std::unordered_map<const as_sketch*, size_t> gi;
  for (int32_t k = 0; k < count; ++k) {
    auto it = gi.find(hs[k]);
    if (it == gi.end()) {
      gi.emplace(hs[k], groups.size());
      groups.push_back({k});
    } else {
      groups[it->second].push_back(k);
    }
  }
  std::vector<as_status> st((size_t)count, AS_OK);
  as::run_parallel((int)groups.size(), [&](int g) {
    as::combined_enter(comb);
    for (int32_t k : groups[(size_t)g]) st[(size_t)k] = as::sk_update_combined(hs[k], rows[k], n[k], ld[k], comb);
    as::combined_leave(comb);
  });
  for (as_status e : st)
    if (e != AS_OK) return e;
  return AS_OK;
}

as_status as_server_create(const as_server_config* cfg, as_server** out) {
  if (!cfg || !out) return AS_EINVAL;
  *out = nullptr;
  const int nw = cfg->workers == 0 ? 16 : cfg->workers;
  if (nw < 1 || nw > 64 || cfg->hbm_budget < 0) return AS_EINVAL;
  as_server* sv = new (std::nothrow) as_server();
  if (!sv) return AS_ENOMEM;
  if (cudaGetDevice(&sv->dev) != cudaSuccess) {
    as_note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
    delete sv;
    return AS_EDEVICE;
  }
  sv->budget = cfg->hbm_budget;
  if (sv->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      as_note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
      delete sv;
      return AS_EDEVICE;
    }
    sv->budget = (int64_t)(0.9 * (double)fr);
  }
  for (int w = 0; w < nw; ++w) sv->workers.emplace_back([sv]() { sv->work(); });
  *out = sv;
  return AS_OK;
}

as_status as_server_open(as_server* sv, const as_config* cfg, double mass_ratio, int64_t* session) {
  if (!sv || !cfg || !session) return AS_EINVAL;
  if (cfg->mode != AS_PERSISTENT || !(mass_ratio >= 1.0) || std::isinf(mass_ratio)) return AS_EINVAL;
  int64_t fp0 = 0;
  as_status st = sketch_footprint(cfg, 0, &fp0);   // validates cfg
  if (st != AS_OK) return st;
  const int32_t ell = cfg->ell > 0 ? cfg->ell : (int32_t)std::ceil(2.0 / cfg->eps);
  const double eps = cfg->eps > 0.0 ? cfg->eps : 2.0 / ell;
  const int64_t rank = attp_rank_bound(eps, mass_ratio);
  int64_t fp = 0;
  st = sketch_footprint(cfg, rank, &fp);
  if (st != AS_OK) return st;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->used + fp > sv->budget) {
      ++sv->refused;
      return AS_EBUSY;
    }
    sv->used += fp;   // held while the session is built
  }
  cudaSetDevice(sv->dev);
  cudaStream_t s = nullptr;
  as_sketch* h = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    as_note_cuda_error(cudaGetLastError(), __FILE__, __LINE__);
    st = AS_EDEVICE;
  }
  if (st == AS_OK) st = sketch_create(cfg, s, &h);
  if (st == AS_OK) st = sketch_reserve(h, rank);
  const int64_t actual = (st == AS_OK) ? std::max<int64_t>(fp, as::sk_device_bytes(h)) : 0;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (st != AS_OK) {
    sv->used -= fp;
    if (h) sketch_destroy(h);
    if (s) cudaStreamDestroy(s);
    return st;
  }
  sv->used += actual - fp;
  const int64_t id = sv->next_session++;
  as_server::Session& S = sv->sessions[id];
  S.h = h;
  S.s = s;
  S.footprint = actual;
  *session = id;
  return AS_OK;
}

as_status as_server_submit(as_server* sv, int64_t session, const float* rows, int64_t n, int64_t ld,
                           int64_t* ticket) {
  if (!sv || n < 0 || (n > 0 && !rows)) return AS_EINVAL;
  const Clock::time_point t0 = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(session);
    if (it == sv->sessions.end()) return AS_EINVAL;
    as_server::Session& S = it->second;
    const int64_t t = sv->next_ticket++;
    as_server::Request& R = sv->reqs[t];
    R.session = session;
    R.rows = rows;
    R.n = n;
    R.ld = ld;
    R.t0 = t0;
    S.pending.push_back(t);
    if (!S.running && S.pending.size() == 1) sv->ready.emplace(t, session);
    ++sv->outstanding;
    if (!sv->have_t0) {
      sv->have_t0 = true;
      sv->first_submit = t0;
    }
    if (ticket) *ticket = t;
  }
  sv->cv_work.notify_one();
  return AS_OK;
}

as_status as_server_wait(as_server* sv, int64_t ticket, double* latency_ms) {
  if (!sv) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return AS_EINVAL;
  sv->cv_done.wait(lk, [&]() {
    auto j = sv->reqs.find(ticket);
    return j == sv->reqs.end() || j->second.done;
  });
  it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return AS_EINVAL;   // forgotten by a concurrent drain
  const as_status st = it->second.st;
  if (latency_ms) *latency_ms = it->second.lat_ms;
  sv->reqs.erase(it);
  return st;
}

as_status as_server_drain(as_server* sv) {
  if (!sv) return AS_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv_done.wait(lk, [&]() { return sv->outstanding == 0; });
  for (auto it = sv->reqs.begin(); it != sv->reqs.end();)
    it = it->second.done ? sv->reqs.erase(it) : std::next(it);
  const as_status st = sv->first_fail;
  sv->first_fail = AS_OK;
  return st;
}

as_status as_server_session(as_server* sv, int64_t session, as_sketch** out) {
  if (!sv || !out) return AS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return AS_EINVAL;
  *out = it->second.h;
  return AS_OK;
}

as_status as_server_close(as_server* sv, int64_t session) {
  if (!sv) return AS_EINVAL;
  as_server::Session S;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(session);
    if (it == sv->sessions.end()) return AS_EINVAL;
    if (it->second.running || !it->second.pending.empty()) return AS_EBUSY;
    S = it->second;
    sv->sessions.erase(it);
    sv->used -= S.footprint;
  }
  sketch_destroy(S.h);
  if (S.s) cudaStreamDestroy(S.s);
  return AS_OK;
}

as_status as_server_stats(as_server* sv, as_server_counters* out) {
  if (!sv || !out) return AS_EINVAL;
  std::vector<double> lat;
  as_server_counters c{};
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    lat = sv->lat;
    c.sessions_open = (int64_t)sv->sessions.size();
    c.sessions_refused = sv->refused;
    c.footprint_bytes = sv->used;
    c.requests_done = sv->done_n;
    c.requests_failed = sv->failed_n;
    c.rows_done = sv->rows_n;
    if (sv->have_t0 && sv->done_n > 0)
      c.span_s = std::max(0.0, std::chrono::duration<double>(sv->last_done - sv->first_submit).count());
  }
  c.p50_ms = percentile(lat, 0.50);
  c.p99_ms = percentile(lat, 0.99);
  double mx = 0.0, sum = 0.0;
  for (double v : lat) {
    mx = std::max(mx, v);
    sum += v;
  }
  c.max_ms = mx;
  c.mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
  *out = c;
  return AS_OK;
}

as_status as_server_reset_stats(as_server* sv) {
  if (!sv) return AS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->lat.clear();
  sv->done_n = sv->failed_n = sv->rows_n = 0;
  sv->have_t0 = false;
  return AS_OK;
}

as_status as_server_destroy(as_server* sv) {
  if (!sv) return AS_OK;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&]() { return sv->outstanding == 0; });
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (std::thread& t : sv->workers) t.join();
  for (auto& kv : sv->sessions) {
    sketch_destroy(kv.second.h);
    if (kv.second.s) cudaStreamDestroy(kv.second.s);
  }
  delete sv;
  return AS_OK;
}

}  // extern "C"
