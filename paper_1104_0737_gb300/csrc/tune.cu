// tune.cu — the autotuner's table and candidate lists (host code only; see
// tune.h).  The GPU timing of the candidates is in dslash.cu.
#include "tune.h"

#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

namespace mbicg {

int TuneTable::pick(const std::string& key, int ncand, const std::function<double(int)>& time, int reps) {
  {
    std::lock_guard<std::mutex> g(mu_);
    auto it = best_.find(key);
    if (it != best_.end()) return it->second;
  }
  // measured outside the lock (the timing launches kernels); two threads that
  // meet a new key at once both measure it and the first to finish wins
  int best = -1;
  double best_t = 0;
  for (int i = 0; i < ncand; ++i) {
    std::vector<double> t;
    for (int r = 0; r < std::max(reps, 1); ++r) {
      const double v = time(i);
      if (v < 0) {
        t.clear();
        break;
      }
      t.push_back(v);
    }
    if (t.empty()) continue;
    std::sort(t.begin(), t.end());
    const double med = t[t.size() / 2];
    if (best < 0 || med < best_t) {
      best = i;
      best_t = med;
    }
  }
  if (best < 0) return -1;
  std::lock_guard<std::mutex> g(mu_);
  return best_.emplace(key, best).first->second;
}

bool TuneTable::lookup(const std::string& key, int* idx) const {
  std::lock_guard<std::mutex> g(mu_);
  auto it = best_.find(key);
  if (it == best_.end()) return false;
  *idx = it->second;
  return true;
}

void TuneTable::set(const std::string& key, int idx) {
  std::lock_guard<std::mutex> g(mu_);
  best_[key] = idx;
}

size_t TuneTable::size() const {
  std::lock_guard<std::mutex> g(mu_);
  return best_.size();
}

int TuneTable::load(const std::string& path) {
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return -1;
  char key[256];
  int idx, n = 0;
  while (fscanf(f, "%255s %d", key, &idx) == 2) {
    set(key, idx);
    ++n;
  }
  fclose(f);
  return n;
}

bool TuneTable::save(const std::string& path) const {
  FILE* f = fopen(path.c_str(), "w");
  if (!f) return false;
  std::lock_guard<std::mutex> g(mu_);
  for (const auto& kv : best_) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
  return fclose(f) == 0;
}

bool autotune_enabled() {
  const char* e = getenv("MBICG_AUTOTUNE");
  return e && e[0] && !(e[0] == '0' && e[1] == 0);
}

TuneTable& tune_table() {
  static TuneTable* t = [] {
    auto* tt = new TuneTable();
    if (const char* p = getenv("MBICG_TUNE_FILE")) tt->load(p);
    return tt;
  }();
  return *t;
}

std::vector<DslashConfig> dslash_candidates(const int dims[4], int L, int max_threads) {
  std::vector<int> sizes;
  for (int S = 1; S * L <= max_threads; S *= 2) sizes.push_back(S);
  std::reverse(sizes.begin(), sizes.end());
  if (sizes.size() > 3) sizes.resize(3);
  const int slice = dims[0] * dims[1] * dims[2];
  std::vector<DslashConfig> out;
  for (int S : sizes) {
    out.push_back({S, 0});
    if (slice % S == 0 && dims[3] % 8 == 0) out.push_back({S, 1});
  }
  return out;
}

std::string dslash_key(int real_bytes, const int dims[4], int L) {
  char b[128];
  snprintf(b, sizeof b, "dslash/fp%d/%dx%dx%dx%d/L%d", real_bytes * 8, dims[0], dims[1], dims[2], dims[3], L);
  return b;
}

std::string sweep_key(bool half, bool clover, const int dims[4], int L) {
  char b[128];
  snprintf(b, sizeof b, "sap_sweep/%s%s/%dx%dx%dx%d/L%d", half ? "fp16" : "fp32", clover ? "/clover" : "", dims[0],
           dims[1], dims[2], dims[3], L);
  return b;
}

}  // namespace mbicg
