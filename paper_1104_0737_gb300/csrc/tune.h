// tune.h — the autotuner's bookkeeping (host code only).  For a key (kernel,
// precision, lattice, columns) it keeps the index of the fastest of a list of
// launch configurations that compute the same result, measured once per
// process (or read from a file named by MBICG_TUNE_FILE) and reused.
#pragma once

#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace mbicg {

class TuneTable {
 public:
  // The chosen configuration for key.  A new key is measured: time(i) gives
  // the milliseconds of one run of candidate i (negative: not usable), called
  // `reps` times per candidate; the smallest median wins (ties: the lower
  // index).  Returns -1 if no candidate is usable (nothing is recorded).
  int pick(const std::string& key, int ncand, const std::function<double(int)>& time, int reps = 3);
  bool lookup(const std::string& key, int* idx) const;
  void set(const std::string& key, int idx);
  size_t size() const;
  // one "key index" line per entry; load() adds to the table and returns the
  // entries read (-1 if the file cannot be opened)
  int load(const std::string& path);
  bool save(const std::string& path) const;

 private:
  mutable std::mutex mu_;
  std::map<std::string, int> best_;
};

TuneTable& tune_table();  // process-wide

// Launch configurations of the operator that give bit-identical results: S
// sites per CTA (one thread per (site, column), S * L <= max_threads, powers
// of two, the three largest) and the CTA order over the lattice (0:
// lexicographic, 1: time slabs of 8 slices, where the segments tile the time
// slices).
struct DslashConfig {
  int S;
  int order;
};
std::vector<DslashConfig> dslash_candidates(const int dims[4], int L, int max_threads);
std::string dslash_key(int real_bytes, const int dims[4], int L);

// Launch shapes of the fused SAP sweep on 8^4 domains; every shape sums each
// column's hops in the same order, so with frozen step lengths (the solver's
// mode) all give bit-identical results (per-column MR sums its dot products
// over the CTAs of a cluster, which differ between shapes: rounding-level
// differences there):
//   0: clusters of 8 CTAs (the domain cut 1x2x2x2, 512 sites per CTA), one
//      column per thread;
//   1: clusters of 16 CTAs (1x2x2x4, 256 sites per CTA), two columns per
//      thread (each link read once for both);
//   2: clusters of 16 CTAs, one column per thread (two CTAs per SM).
constexpr int SWEEP_SHAPES = 3;
// half: FP16 storage of the residual and psi; clover: the Jacobi-preconditioned
// clover operator
std::string sweep_key(bool half, bool clover, const int dims[4], int L);

}  // namespace mbicg
