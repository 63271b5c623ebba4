// P5 (Algorithm 10): the tracking distributed matrix sketch with m sites and
// one coordinator, driven in synchronous rounds on one stream.
//
// Site j, for each of its rows a (in order):
//   F_j += ||a||^2; if F_j >= (eps/m) F_hat_known: message F_j, F_j = 0;
//   AeroSketch update of a (AS_SITE sketch, threshold theta);
//   every snapshot taken is sent to the coordinator and deleted.
// Coordinator:
//   each message: F_hat += F_j, msgs += 1; at msgs >= m: msgs = 0 and
//   broadcast F_hat (every site then uses theta = (eps/m) F_hat);
//   each snapshot (Z, Y = Z^T C'^T C'): B += Z Y + Y^T Z^T - Z (Y Z) Z^T;
//   Query: the eigen-shrink of Algorithm 5 on B.
// Readings: a site starts with theta = +inf (Algorithm 10 leaves the initial
// threshold open; with 0 the stop test of Algorithm 2 would depend on the
// rounding sign of numerically zero Ritz values), its threshold after a
// broadcast is (eps/m) F_hat (the per-site error of the analysis), and the
// messages of a round reach the coordinator at the round's end in site order.
//
// The scalar protocol runs on the host; the rows, the snapshot terms and the
// coordinator's query run in the library's kernels (sketch calls only).  Each
// site has its own stream, and a round updates the sites from the library's
// worker threads so that their kernels overlap on the GPU.
#include <algorithm>
#include <cmath>
#include <new>
#include <thread>
#include <vector>

#include "kernels.cuh"

struct as_p5 {
  int m = 0, d = 0, ell = 0;
  double eps = 0.0;
  cudaStream_t s = nullptr;
  std::vector<as_sketch*> sites;
  std::vector<cudaStream_t> ss;   // one stream per site: sites update concurrently
  as_sketch* coord = nullptr;
  std::vector<double> F;     // unsent row mass of each site
  double F_site = 0.0;       // F_hat as the sites know it (last broadcast)
  double F_hat = 0.0;        // the coordinator's running sum
  int msgs = 0;
  as_p5_counters st{};
};

extern "C" {

as_status as_p5_destroy(as_p5* p) {
  if (!p) return AS_OK;
  for (as_sketch* h : p->sites) sketch_destroy(h);
  sketch_destroy(p->coord);
  for (cudaStream_t s : p->ss) cudaStreamDestroy(s);
  delete p;
  return AS_OK;
}

as_status as_p5_create(const as_config* site_cfg, int32_t m, void* cuda_stream, as_p5** out) {
  if (!site_cfg || !out || m < 1) return AS_EINVAL;
  *out = nullptr;
  as_p5* p = new (std::nothrow) as_p5();
  if (!p) return AS_ENOMEM;
  p->m = m;
  p->s = (cudaStream_t)cuda_stream;
  as_config c = *site_cfg;
  c.mode = AS_COORDINATOR;
  as_status st = sketch_create(&c, cuda_stream, &p->coord);
  for (int j = 0; j < m && st == AS_OK; ++j) {
    as_config cj = *site_cfg;
    cj.mode = AS_SITE;
    cj.theta = INFINITY;
    cj.stream_id = site_cfg->stream_id + (uint64_t)j;
    as_sketch* h = nullptr;
    cudaStream_t sj = nullptr;
    if (cudaStreamCreateWithFlags(&sj, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = AS_EDEVICE;
      break;
    }
    p->ss.push_back(sj);
    st = sketch_create(&cj, sj, &h);
    if (st == AS_OK) p->sites.push_back(h);
  }
  if (st == AS_OK) {
    as_stats cs{};
    st = sketch_stats(p->coord, &cs);
    p->d = cs.d;
    p->ell = cs.ell;
    p->eps = (site_cfg->eps > 0.0) ? site_cfg->eps : 2.0 / cs.ell;
  }
  if (st != AS_OK) {
    as_p5_destroy(p);
    return st;
  }
  p->F.assign((size_t)m, 0.0);
  *out = p;
  return AS_OK;
}

as_status as_p5_round(as_p5* p, const float* const* rows, const int64_t* n, const int64_t* ld) {
  if (!p || !rows || !n || !ld) return AS_EINVAL;
  for (int j = 0; j < p->m; ++j)
    if (n[j] < 0 || (n[j] > 0 && (!rows[j] || ld[j] < p->d))) return AS_EINVAL;
  // the sites' rows, each site on its own stream and a worker thread: row
  // norms for the protocol and the site update.  The sites progress
  // independently: sharing launches of the batched iterations (lockstep
  // blocks, or the launch combiner of sketch_update_grouped) measured slower
  // here, since a shared launch waits for the slowest site's decisions.
  const int m = p->m;
  std::vector<std::vector<double>> nrm((size_t)m);
  std::vector<as_status> sts((size_t)m, AS_OK);
  as::run_parallel(m, [&](int j) {
    nrm[(size_t)j].assign((size_t)n[j], 0.0);
    sts[(size_t)j] = as::row_norms_f64(rows[j], n[j], ld[j], p->d, p->ss[(size_t)j], nrm[(size_t)j].data());
    if (sts[(size_t)j] == AS_OK && n[j] > 0) sts[(size_t)j] = sketch_update(p->sites[(size_t)j], rows[j], n[j], ld[j]);
  });
  for (as_status st : sts)
    if (st != AS_OK) return st;
  // messages and snapshots in site order (the coordinator's sums keep a fixed order)
  std::vector<double> pending;
  for (int j = 0; j < m; ++j) {
    for (double v : nrm[(size_t)j]) {
      p->F[(size_t)j] += v;
      if (p->F[(size_t)j] >= (p->eps / p->m) * p->F_site) {   // message F_j
        pending.push_back(p->F[(size_t)j]);
        p->F[(size_t)j] = 0.0;
      }
    }
    int32_t sent = 0;
    as_status st = sketch_send_snapshots(p->sites[(size_t)j], p->coord, &sent);
    if (st != AS_OK) return st;
    p->st.snapshots_sent += sent;
  }
  for (double f : pending) {   // the coordinator's Receive_Update, at the round's end
    p->F_hat += f;
    p->st.messages += 1;
    if (++p->msgs >= p->m) {
      p->msgs = 0;
      p->st.broadcasts += 1;
      p->F_site = p->F_hat;
      for (as_sketch* h : p->sites) {
        as_status st = sketch_set_theta(h, (p->eps / p->m) * p->F_hat);
        if (st != AS_OK) return st;
      }
    }
  }
  p->st.rounds += 1;
  p->st.f_hat = p->F_hat;
  p->st.f_site = p->F_site;
  return AS_OK;
}

as_status as_p5_query(as_p5* p, float* out, int64_t ldo, int32_t* rows_out) {
  if (!p) return AS_EINVAL;
  return sketch_query(p->coord, -1, out, ldo, rows_out);
}

as_status as_p5_query_gram(as_p5* p, double* out) {
  if (!p) return AS_EINVAL;
  return sketch_query_gram(p->coord, -1, out);
}

as_status as_p5_stats(as_p5* p, as_p5_counters* out) {
  if (!p || !out) return AS_EINVAL;
  *out = p->st;
  return AS_OK;
}

as_status as_p5_site(as_p5* p, int32_t j, as_sketch** out) {
  if (!p || !out || j < 0 || j >= p->m) return AS_EINVAL;
  *out = p->sites[(size_t)j];
  return AS_OK;
}

as_status as_p5_coordinator(as_p5* p, as_sketch** out) {
  if (!p || !out) return AS_EINVAL;
  *out = p->coord;
  return AS_OK;
}

}  // extern "C"
