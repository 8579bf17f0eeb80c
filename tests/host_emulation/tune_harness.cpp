// C entry points over the autotuner's host code (tune.cu, compiled with g++)
// for the CPU tests: the table with a scripted timer, and the candidate list.
#include "tune.h"

#include <cstring>
#include <thread>

using namespace mbicg;

static TuneTable table;
static const double* g_times = nullptr;  // scripted: g_times[i * reps + r]
static int g_reps = 1, g_calls = 0;

extern "C" {
int tune_pick(const char* key, int ncand, const double* times, int reps) {
  g_times = times;
  g_reps = reps;
  int call[64] = {0};
  return table.pick(key, ncand, [&](int i) {
    ++g_calls;
    return g_times[i * g_reps + call[i]++];
  }, reps);
}
int tune_calls() { return g_calls; }
int tune_size() { return (int)table.size(); }
int tune_save(const char* path) { return table.save(path) ? 1 : 0; }
int tune_load(const char* path) { return table.load(path); }
int tune_lookup(const char* key) {
  int idx = -2;
  return table.lookup(key, &idx) ? idx : -2;
}
// picks on nkeys distinct keys from nthreads threads at once; returns the table size
int tune_concurrent(int nthreads, int nkeys) {
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([t, nkeys] {
      for (int k = 0; k < nkeys; ++k) {
        const std::string key = "c/" + std::to_string(k);
        table.pick(key, 3, [k](int i) { return (double)((i + k) % 3); }, 1);
      }
    });
  for (auto& x : th) x.join();
  return (int)table.size();
}
// candidates: writes (S, order) pairs, returns the count
int tune_candidates(const int* dims, int L, int max_threads, int* out) {
  const auto c = dslash_candidates(dims, L, max_threads);
  for (size_t i = 0; i < c.size(); ++i) {
    out[2 * i] = c[i].S;
    out[2 * i + 1] = c[i].order;
  }
  return (int)c.size();
}
int tune_key(int real_bytes, const int* dims, int L, char* buf, int n) {
  const std::string k = dslash_key(real_bytes, dims, L);
  strncpy(buf, k.c_str(), n);
  return (int)k.size();
}
int tune_sweep_key(int half, int clover, const int* dims, int L, char* buf, int n) {
  const std::string k = sweep_key(half != 0, clover != 0, dims, L);
  strncpy(buf, k.c_str(), n);
  return (int)k.size();
}
int tune_sweep_shapes() { return SWEEP_SHAPES; }
}
