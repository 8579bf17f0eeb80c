// Threaded host emulation shim: every CUDA thread of a launch runs as its own
// host thread, so kernels that synchronise (__syncthreads, cluster barriers,
// warp shuffles) and share on-chip memory (shared memory, distributed shared
// memory of a thread-block cluster) can run on the CPU.  Shared memory is one
// arena per CTA, filled with NaN bytes before the launch so that a read of a
// word no thread has written shows up in the result.
#pragma once
#include <cuda_runtime.h>
#include <pthread.h>

#include <barrier>
#include <optional>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <unordered_map>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <memory>
#include <semaphore>
#include <vector>
#if defined(__SANITIZE_ADDRESS__)
#include <sanitizer/asan_interface.h>
#endif

struct EmuDim {
  unsigned x, y, z;
};

struct EmuCta {
  std::vector<unsigned char> arena;  // dynamic shared memory, then the static variables
  size_t dyn_bytes = 0;
  std::unique_ptr<std::barrier<>> bar;
  std::vector<std::unique_ptr<std::barrier<>>> warp_bar;
  std::vector<unsigned long long> warp_slot;
  int or_flag = 0;
};

struct EmuCluster {
  std::vector<EmuCta*> ctas;
  std::unique_ptr<std::barrier<>> bar;
};

struct EmuThread {
  EmuDim block, thread;
  EmuCta* cta;
  EmuCluster* cluster;
  unsigned rank;
};

extern thread_local EmuThread emu_t;
extern EmuDim blockDim, gridDim;
// set when an emulated access leaves the cluster or a CTA's arena (the access
// reads NaN or CTA 0 instead); the harness reports it
extern int emu_bad_access;
#define blockIdx (emu_t.block)
#define threadIdx (emu_t.thread)

template <typename T>
inline T __ldg(const T* p) { return *p; }
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
inline size_t __cvta_generic_to_shared(const void* p) {
  return (size_t)((const unsigned char*)p - emu_t.cta->arena.data());
}
inline void __syncthreads() { emu_t.cta->bar->arrive_and_wait(); }
inline int atomicOr(int* p, int v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }

template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int o) {
  static_assert(sizeof(T) <= 8, "shuffle of a type wider than 8 bytes");
  const unsigned tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const unsigned w = tid / 32, lane = tid % 32;
  unsigned long long bits = 0;
  memcpy(&bits, &v, sizeof(T));
  emu_t.cta->warp_slot[w * 32 + lane] = bits;
  emu_t.cta->warp_bar[w]->arrive_and_wait();
  const unsigned long long rb = emu_t.cta->warp_slot[w * 32 + (lane ^ (unsigned)o)];
  emu_t.cta->warp_bar[w]->arrive_and_wait();
  T r;
  memcpy(&r, &rb, sizeof(T));
  return r;
}

// Static __shared__ variables: the source cutter gives each declaration of the
// emulated code its own slot of EMU_SLOT_BYTES after the dynamic part.
#ifndef EMU_STATIC_SLOTS
#define EMU_STATIC_SLOTS 1
#endif
constexpr size_t EMU_SLOT_BYTES = 8192;
// under AddressSanitizer a poisoned gap follows the dynamic part (and the
// arena), so that a kernel's access past its dynamic shared memory is reported
#if defined(__SANITIZE_ADDRESS__)
constexpr size_t EMU_SMEM_REDZONE = 256;
#else
constexpr size_t EMU_SMEM_REDZONE = 0;
#endif
inline void* emu_dyn_smem() { return emu_t.cta->arena.data(); }
inline void* emu_static_smem_slot(int i) {
  return emu_t.cta->arena.data() + emu_t.cta->dyn_bytes + EMU_SMEM_REDZONE + (size_t)i * EMU_SLOT_BYTES;
}
inline int __syncthreads_or(int p);

namespace cooperative_groups {
struct cluster_group {
  unsigned block_rank() const { return emu_t.rank; }
  void sync() const { emu_t.cluster->bar->arrive_and_wait(); }
  template <typename T>
  T* map_shared_rank(T* p, unsigned r) const;
};
inline cluster_group this_cluster() { return {}; }
}  // namespace cooperative_groups

template <typename T>
T* cooperative_groups::cluster_group::map_shared_rank(T* p, unsigned r) const {
  const size_t off = (size_t)((unsigned char*)p - emu_t.cta->arena.data());
  if (r >= emu_t.cluster->ctas.size() || off >= emu_t.cta->arena.size()) {
    __atomic_store_n(&emu_bad_access, 1, __ATOMIC_SEQ_CST);
    r = 0;
  }
  return reinterpret_cast<T*>(emu_t.cluster->ctas[r]->arena.data() + off);
}

// the two halves of the cluster barrier: the arrival of this emulated thread
// is held between them
inline thread_local std::optional<std::barrier<>::arrival_token> emu_cluster_token;
inline void emu_cluster_arrive() { emu_cluster_token.emplace(emu_t.cluster->bar->arrive()); }
inline void emu_cluster_wait() {
  emu_t.cluster->bar->wait(std::move(*emu_cluster_token));
  emu_cluster_token.reset();
}

// shared::cluster window addresses: the CTA rank in the top 8 bits, the
// offset in the CTA's arena below; mapa of a window address replaces the rank
inline uint32_t emu_mapa(uint32_t addr, uint32_t rank) { return (rank << 24) | (addr & 0xffffffu); }
inline float4 emu_ld_cluster_f4(uint32_t a) {
  const uint32_t r = a >> 24, off = a & 0xffffffu;
  if (r >= emu_t.cluster->ctas.size() || (size_t)off + 16 > emu_t.cluster->ctas[r]->arena.size()) {
    __atomic_store_n(&emu_bad_access, 1, __ATOMIC_SEQ_CST);
    const float n = std::nanf("");
    return make_float4(n, n, n, n);
  }
  float4 v;
  memcpy(&v, emu_t.cluster->ctas[r]->arena.data() + off, 16);
  return v;
}

#define __launch_bounds__(...)
using std::fma;
using std::isfinite;
using std::isnan;
// sin(pi x) and cos(pi x)
inline void sincospi(double x, double* s, double* c) {
  *s = std::sin(M_PI * x);
  *c = std::cos(M_PI * x);
}

inline int __syncthreads_or(int p) {
  EmuCta* c = emu_t.cta;
  emu_t.cta->bar->arrive_and_wait();  // the previous use of the flag is over
  if (p) __atomic_store_n(&c->or_flag, 1, __ATOMIC_SEQ_CST);
  c->bar->arrive_and_wait();
  const int r = __atomic_load_n(&c->or_flag, __ATOMIC_SEQ_CST);
  c->bar->arrive_and_wait();
  if (threadIdx.x == 0) __atomic_store_n(&c->or_flag, 0, __ATOMIC_SEQ_CST);
  return r;
}

// mbarrier and bulk-copy emulation: the barrier's state lives in a side table
// keyed by its shared-memory address; a bulk copy is a memcpy that then
// completes its bytes on the barrier.  A phase completes when its arrivals
// and its expected transaction bytes are both done.  A wait sleeps on a
// condition variable; one that sees no progress for two seconds gives up, and
// from then on every wait of the launch gives up at once (the kernel's own
// path for a copy that never completes).
struct EmuMbar {
  int expected = 0, pending = 0;
  long long tx = 0;
  unsigned phases = 0;  // completed phases
};
struct EmuMbarTable {
  std::mutex mu;
  std::condition_variable cv;
  std::unordered_map<const void*, EmuMbar> tab;
  bool gave_up = false;
};
inline EmuMbarTable& emu_mbars() {
  static EmuMbarTable t;
  return t;
}
inline void emu_mbar_settle(EmuMbar& b) {
  if (b.pending == 0 && b.tx == 0) {
    ++b.phases;
    b.pending = b.expected;
  }
}
inline void emu_mbar_init(const void* bar, int count) {
  auto& t = emu_mbars();
  std::lock_guard<std::mutex> g(t.mu);
  EmuMbar& b = t.tab[bar];
  b = EmuMbar{};
  b.expected = b.pending = count;
}
// an arrival (tx_add extra transaction bytes expected) or completed bytes (done)
inline void emu_mbar_update(const void* bar, int arrivals, long long tx_add, long long done) {
  auto& t = emu_mbars();
  {
    std::lock_guard<std::mutex> g(t.mu);
    EmuMbar& b = t.tab[bar];
    b.tx += tx_add - done;
    b.pending -= arrivals;
    emu_mbar_settle(b);
  }
  t.cv.notify_all();
}
inline bool emu_mbar_try(const void* bar, uint32_t parity) {
  auto& t = emu_mbars();
  std::lock_guard<std::mutex> g(t.mu);
  return (t.tab[bar].phases & 1u) != (parity & 1u);
}
inline bool emu_mbar_wait(const void* bar, uint32_t parity) {
  auto& t = emu_mbars();
  std::unique_lock<std::mutex> g(t.mu);
  if (t.gave_up) return false;
  const bool ok = t.cv.wait_for(g, std::chrono::seconds(2), [&] {
    return t.gave_up || (t.tab[bar].phases & 1u) != (parity & 1u);
  });
  if (!ok || t.gave_up) {
    t.gave_up = true;
    t.cv.notify_all();
    return false;
  }
  return true;
}
inline void emu_mbar_reset() {
  auto& t = emu_mbars();
  std::lock_guard<std::mutex> g(t.mu);
  t.tab.clear();
  t.gave_up = false;
}
inline long long min(long long a, long long b) { return a < b ? a : b; }

// Host threads that run the CUDA threads of one cluster at a time, all at
// once (they meet at the emulated barriers).  Created on first use, 512 KB of
// stack each, and reused by every later launch: creating a thread per CUDA
// thread per launch dominated the emulation's run time.  One launch at a time.
class EmuPool {
 public:
  static EmuPool& get() {
    static EmuPool* p = new EmuPool();  // never destroyed: its threads wait until the process ends
    return *p;
  }
  // fn(ctx, i) for i < n, each on its own thread; returns when all have returned
  void run(size_t n, void (*fn)(void*, size_t), void* ctx) {
    std::lock_guard<std::mutex> g(launch_mu_);
    while (workers_.size() < n) add_worker();
    fn_ = fn;
    ctx_ = ctx;
    left_.store(n, std::memory_order_relaxed);
    for (size_t i = 0; i < n; ++i) workers_[i]->go.release();
    if (n) done_.acquire();
  }

 private:
  struct Worker {
    EmuPool* pool;
    size_t index;
    std::binary_semaphore go{0};
  };
  static void* loop(void* p) {
    Worker* w = static_cast<Worker*>(p);
    EmuPool* pool = w->pool;
    for (;;) {
      w->go.acquire();
      pool->fn_(pool->ctx_, w->index);
      if (pool->left_.fetch_sub(1, std::memory_order_acq_rel) == 1) pool->done_.release();
    }
    return nullptr;
  }
  void add_worker() {
    auto w = std::make_unique<Worker>();
    w->pool = this;
    w->index = workers_.size();
    pthread_attr_t attr;
    pthread_attr_init(&attr);
    pthread_attr_setstacksize(&attr, 1 << 19);
    pthread_attr_setdetachstate(&attr, PTHREAD_CREATE_DETACHED);
    pthread_t tid;
    const int rc = pthread_create(&tid, &attr, &EmuPool::loop, w.get());
    pthread_attr_destroy(&attr);
    if (rc != 0) {  // a missing thread would leave the others waiting at a barrier
      fprintf(stderr, "emu_launch: pthread_create failed (%d)\n", rc);
      abort();
    }
    workers_.push_back(std::move(w));
  }
  std::mutex launch_mu_;
  std::vector<std::unique_ptr<Worker>> workers_;
  void (*fn_)(void*, size_t) = nullptr;
  void* ctx_ = nullptr;
  std::atomic<size_t> left_{0};
  std::binary_semaphore done_{0};
};

// Runs kernel() for a grid of nclusters clusters of cs CTAs of `threads`
// threads each (1-D), one cluster at a time; the static slots follow
// dyn_bytes of dynamic shared memory in each CTA's arena.
template <typename F>
void emu_launch3(int nclusters, int cs, dim3 block, size_t dyn_bytes, F kernel);
template <typename F>
void emu_launch(int nclusters, int cs, int threads, size_t dyn_bytes, F kernel) {
  emu_launch3(nclusters, cs, dim3((unsigned)threads, 1, 1), dyn_bytes, kernel);
}
// as emu_launch, with a 3-D CTA shape (thread t has x = t % block.x fastest)
// one launch at a time, also when several host threads launch (blockDim and
// gridDim are process-wide)
inline std::mutex& emu_launch_mutex() {
  static std::mutex m;
  return m;
}
template <typename F>
void emu_launch3(int nclusters, int cs, dim3 block, size_t dyn_bytes, F kernel) {
  std::lock_guard<std::mutex> launch_lock(emu_launch_mutex());
  emu_mbar_reset();  // a wait that gave up in an earlier launch does not end this one's
  const int threads = (int)(block.x * block.y * block.z);
  const size_t static_bytes = (size_t)EMU_STATIC_SLOTS * EMU_SLOT_BYTES;
  blockDim = {block.x, block.y, block.z};
  gridDim = {(unsigned)(nclusters * cs), 1, 1};
  for (int cl = 0; cl < nclusters; ++cl) {
    EmuCluster cluster;
    std::vector<std::unique_ptr<EmuCta>> ctas;
    for (int r = 0; r < cs; ++r) {
      auto c = std::make_unique<EmuCta>();
      c->arena.assign(dyn_bytes + EMU_SMEM_REDZONE + static_bytes + 16, 0xff);
      c->dyn_bytes = dyn_bytes;
#if defined(__SANITIZE_ADDRESS__)
      ASAN_POISON_MEMORY_REGION(c->arena.data() + dyn_bytes, EMU_SMEM_REDZONE);
      ASAN_POISON_MEMORY_REGION(c->arena.data() + dyn_bytes + EMU_SMEM_REDZONE + static_bytes, 16);
#endif
      c->bar = std::make_unique<std::barrier<>>(threads);
      for (int w = 0; w < (threads + 31) / 32; ++w) c->warp_bar.push_back(std::make_unique<std::barrier<>>(32));
      c->warp_slot.assign((size_t)((threads + 31) / 32) * 32, 0);
      cluster.ctas.push_back(c.get());
      ctas.push_back(std::move(c));
    }
    cluster.bar = std::make_unique<std::barrier<>>(cs * threads);
    struct Arg {
      EmuThread t;
      F* k;
    };
    std::vector<Arg> args((size_t)cs * threads);
    for (int r = 0; r < cs; ++r)
      for (int t = 0; t < threads; ++t) {
        Arg& a = args[(size_t)r * threads + t];
        const unsigned tx = (unsigned)t % block.x, ty = ((unsigned)t / block.x) % block.y,
                       tz = (unsigned)t / (block.x * block.y);
        a.t = EmuThread{{(unsigned)(cl * cs + r), 0, 0}, {tx, ty, tz}, ctas[r].get(), &cluster, (unsigned)r};
        a.k = &kernel;
      }
    EmuPool::get().run(args.size(), [](void* p, size_t i) {
      Arg& a = static_cast<Arg*>(p)[i];
      emu_t = a.t;
      (*a.k)();
    }, args.data());
  }
}
