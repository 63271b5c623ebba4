// Launch-shape autotuner keyed by problem shape.
//
// A kernel with several valid launch shapes (lanes per item, K splits, slab
// widths) asks tune_pick for one.  The first call for a (device, kernel, key)
// times every candidate on that call's own inputs (CUDA events on the
// caller's stream, after one untimed run of each), keeps the fastest and, if
// it was not the last candidate run, runs it once more so that the call's
// outputs are the winner's.  Every later call with the same key gets the
// cached choice without timing.  The key is the problem shape only, so a
// sketch's results do not depend on which other sketches run beside it; they
// can differ between processes when two candidates time alike, and
// AS_TUNE=0 in the environment turns tuning off (the first candidate, the
// default shape, is used everywhere).  A candidate whose run returns
// AS_ENOTSUP (a shape the device cannot hold) is skipped.
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "kernels.cuh"

namespace as {

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, std::string, long long>, int> g_tuned;

bool tuning_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("AS_TUNE");
    return !(v && v[0] == '0');
  }();
  return on;
}

}  // namespace

int tune_pick(cudaStream_t s, const char* kernel, long long key, const int* choices, int n,
              const std::function<as_status(int)>& run, as_status* st, bool* ran) {
  *st = AS_OK;
  *ran = false;
  if (n <= 1 || !tuning_enabled()) return choices[0];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return choices[0];
  }
  // one tuning at a time: a concurrent caller with the same key waits and
  // then finds the cached choice
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto k = std::make_tuple(dev, std::string(kernel), key);
  auto it = g_tuned.find(k);
  if (it != g_tuned.end()) return it->second;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    (void)cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return choices[0];
  }
  int best = -1, last = -1;
  float best_ms = 0.f;
  for (int c = 0; c < n && *st == AS_OK; ++c) {
    *st = run(choices[c]);   // untimed: first-launch costs (module loading, attributes)
    if (*st == AS_ENOTSUP) {   // a shape this device cannot run: skip it
      *st = AS_OK;
      continue;
    }
    if (*st != AS_OK) break;
    cudaEventRecord(e0, s);
    *st = run(choices[c]);
    cudaEventRecord(e1, s);
    last = c;
    if (*st != AS_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      (void)cudaGetLastError();
      *st = AS_EDEVICE;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*st == AS_OK && best < 0) *st = AS_ENOTSUP;   // no candidate could run
  if (*st != AS_OK) return choices[0];
  g_tuned[k] = choices[best];
  if (best == last) {
    *ran = true;
  } else {
    *st = run(choices[best]);
    *ran = (*st == AS_OK);
  }
  return choices[best];
}

}  // namespace as
