// serve.cu — a request loop over resident gauge fields.
//
// Requests are source blocks of 1..12 columns for one of several resident
// gauge fields and a hopping parameter.  Each field has solver slots (a
// solver context with its own CUDA stream and host thread, holding the
// field's links); a free slot takes the oldest waiting request of its field
// and packs behind it, in arrival order, the waiting requests with the same
// kappa and tolerance that still fit into one block of at most 12 columns;
// the packed block is solved by the modified block BiCGSTAB (Algorithm 2 of
// Sec. 2.1 — the method solves the L columns of a block together) and the
// columns are handed back to their requests.
//
// Admission by HBM footprint: the server holds a device-memory budget.  The
// slots' links are charged when a field is added; a packed block is admitted
// only when the workspace of its block solve (the solver's blocks at its L,
// the packing buffers) fits beside everything already held, and packing stops
// at the request that would not fit.  A slot keeps its workspace between
// solves (charged while held); when a slot cannot admit even the oldest
// request, idle slots give their workspaces back, and if that is not enough
// it waits for a running solve to finish; with no solve running, the request
// can never be admitted (fields added after it took the budget) and ends with
// MBICG_ENOMEM.  Slots of different fields, and
// several slots of one field, run their solves concurrently on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mbicg.h"
#include "internal.h"

using namespace mbicg;

namespace {

constexpr int SERVE_MAXL = 12;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// columns [o, o + Lj) of the packed block (L columns) <-> a request's block
// (Lj columns); both in the ABI layout [site][spin*colour][column]
__global__ void k_pack_columns(long long nrow, int L, int o, int Lj, const cx<double>* __restrict__ in,
                               cx<double>* __restrict__ out, int to_packed) {
  const long long n = nrow * Lj;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / Lj;
    const int j = (int)(i - row * Lj);
    if (to_packed)
      out[row * L + o + j] = in[i];
    else
      out[i] = in[row * L + o + j];
  }
}

struct Request {
  long long id = 0;
  int field = 0, L = 0;
  double kappa = 0, tol = 0;
  std::vector<double> B, X;  // ABI layout, interleaved complex
  std::vector<double> tres;
  int status = 1, iters = 0, batch_cols = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  bool done = false;
  bool claimed = false;  // a wait has taken it: any other wait for it is refused
};

struct Slot {
  int field = 0;
  long long V = 0;        // the field's sites and solver parameters, copied so that
  mbicg_params params{};  // a running solve never reads the server's field list
  mbicg_ctx* ctx = nullptr;
  cx<double>* dB = nullptr;  // packed block
  cx<double>* dX = nullptr;
  cx<double>* dS = nullptr;  // one request's columns
  int cap = 0;               // columns the packing buffers hold
  double held = 0;           // bytes of workspace charged to this slot (beyond its links)
  bool busy = false;
  std::thread th;
};

struct Field {
  int dims[4] = {0, 0, 0, 0};
  long long V = 0;
  mbicg_params params{};
  int nslots = 0;
};

}  // namespace

struct mbicg_server {
  int device = 0;
  double budget = 0, used = 0;  // bytes
  long long mem_waits = 0;      // block solves that waited for memory
  std::vector<Field> fields;
  std::vector<Slot*> slots;
  std::mutex add_mu;  // one mbicg_server_add_field at a time
  std::deque<Request*> pending;
  std::map<long long, Request*> requests;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  bool hold = false;  // while set, no slot starts a new block solve
  long long next_id = 1;
  long long solves = 0, columns = 0, max_cols = 0;
};

namespace {

// Device bytes a slot of a field holds for the links (FP64, FP32, the FP16
// rows and the FP32 rows) and its fixed scratch.
double slot_fixed_bytes(long long V) { return V * (576.0 + 288 + 96 + 192) + (1 << 22); }

// Device bytes of the workspace of a block solve of L columns on V sites: B,
// X and W in FP64, the seven Krylov blocks, the preconditioner's blocks (FP32
// r, q, x; the FP16 storage on top when chosen), the packing buffers (packed
// B and X, one request's columns) and the small per-CTA partial sums; 5 %
// margin.
double solve_bytes(long long V, int L, const mbicg_params& p) {
  const double nl = 12.0 * V * L;
  double b = 3 * 16 * nl;                                  // B64, X64, W64
  b += 7 * (p.prec_D == MBICG_FP64 ? 16 : 8) * nl;         // R, P, R~, U, V, S, Z
  if (p.ncycle > 0) {
    const double sap = p.prec_sap == MBICG_FP64 ? 16 : 8;
    b += 3 * sap * nl;                                     // SAP r, q, x
    if ((p.prec_sap == MBICG_FP64) != (p.prec_D == MBICG_FP64)) b += 2 * sap * nl;  // eta, psi staging
    if (p.prec_sap == MBICG_FP16) b += 3 * (4 * nl + 4.0 * V * L);
  }
  b += 3 * 16 * nl;                                        // packing buffers
  return 1.05 * b + (8 << 20);
}

// Bytes a slot holds now: its context's workspaces and its packing buffers.
double slot_held_bytes(const Slot* sl, long long V) {
  return (double)ctx_workspace_bytes(sl->ctx) + 3.0 * sizeof(cx<double>) * V * 12 * sl->cap;
}

void release_slot_workspace(mbicg_server* s, Slot* sl) {
  ctx_release_workspace(sl->ctx);
  if (sl->dB) cudaFree(sl->dB);
  if (sl->dX) cudaFree(sl->dX);
  if (sl->dS) cudaFree(sl->dS);
  sl->dB = sl->dX = sl->dS = nullptr;
  sl->cap = 0;
  s->used -= sl->held;
  sl->held = 0;
}

// Takes the oldest waiting request of `field` and the compatible ones behind
// it that fit into 12 columns and into the memory budget (the slot's own
// workspace counts as available to it); charges the batch's workspace to the
// slot.  *no_memory: the oldest request did not fit.  Called with s->mu held.
std::vector<Request*> take_batch(mbicg_server* s, Slot* sl, bool* no_memory) {
  const Field& f = s->fields[sl->field];
  std::vector<Request*> batch;
  int cols = 0;
  *no_memory = false;
  const double avail = s->budget - s->used + sl->held;
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request* r = *it;
    const bool compatible = r->field == sl->field && cols + r->L <= SERVE_MAXL &&
                            (batch.empty() || (r->kappa == batch[0]->kappa && r->tol == batch[0]->tol));
    if (!compatible) {
      ++it;
      continue;
    }
    if (solve_bytes(f.V, cols + r->L, f.params) > avail) {
      if (batch.empty()) *no_memory = true;
      break;  // later requests wait behind it: arrival order is kept
    }
    batch.push_back(r);
    cols += r->L;
    it = s->pending.erase(it);
  }
  if (!batch.empty()) {
    const double need = solve_bytes(f.V, cols, f.params);
    if (need > sl->held) {
      s->used += need - sl->held;
      sl->held = need;
    }
  }
  return batch;
}

// Called without s->mu: the fields' list may grow meanwhile (another
// mbicg_server_add_field), so only the slot's own copy of its field is read.
void run_batch(mbicg_server* s, Slot* sl, std::vector<Request*>& batch) {
  const long long nrow = sl->V * 12;
  int L = 0;
  for (Request* r : batch) L += r->L;
  const double t0 = now_ms();
  for (Request* r : batch) r->t_start = t0;
  cudaStream_t st = nullptr;
  int status = MBICG_OK, iters = 0;
  double tres[MAXL] = {0};
  cudaSetDevice(s->device);
  if (sl->cap < L) {
    // packing buffers for L columns (the previous ones are too small)
    if (sl->dB) cudaFree(sl->dB);
    if (sl->dX) cudaFree(sl->dX);
    if (sl->dS) cudaFree(sl->dS);
    sl->dB = sl->dX = sl->dS = nullptr;
    sl->cap = 0;
    const size_t blk = sizeof(cx<double>) * (size_t)nrow * L;
    if (cudaMalloc(&sl->dB, blk) != cudaSuccess || cudaMalloc(&sl->dX, blk) != cudaSuccess ||
        cudaMalloc(&sl->dS, blk) != cudaSuccess) {
      cudaGetLastError();
      status = MBICG_ENOMEM;
    } else {
      sl->cap = L;
    }
  }
  if (status == MBICG_OK) {
    // the stream of the slot's context is its own non-blocking stream
    st = ctx_stream(sl->ctx);
    int o = 0;
    for (Request* r : batch) {
      if (cudaMemcpyAsync(sl->dS, r->B.data(), sizeof(cx<double>) * nrow * r->L, cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        status = MBICG_ECUDA;
      k_pack_columns<<<1024, 256, 0, st>>>(nrow, L, o, r->L, sl->dS, sl->dB, 1);
      o += r->L;
    }
    if (status == MBICG_OK && cudaGetLastError() != cudaSuccess) status = MBICG_ECUDA;
  }
  if (status == MBICG_OK)
    status = mbicg_block_solve(sl->ctx, reinterpret_cast<const double*>(sl->dB), reinterpret_cast<double*>(sl->dX),
                               L, batch[0]->kappa, batch[0]->tol, &sl->params, &iters, tres);
  const bool have_x = status == MBICG_OK || status == MBICG_ENOTCONV || status == MBICG_EBREAKDOWN;
  int o = 0;
  for (Request* r : batch) {
    r->X.assign(2 * (size_t)nrow * r->L, 0.0);
    r->tres.assign(r->L, 0.0);
    if (have_x && st) {
      k_pack_columns<<<1024, 256, 0, st>>>(nrow, L, o, r->L, sl->dX, sl->dS, 0);
      if (cudaMemcpyAsync(r->X.data(), sl->dS, sizeof(cx<double>) * nrow * r->L, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        status = MBICG_ECUDA;
      for (int j = 0; j < r->L; ++j) r->tres[j] = tres[o + j];
    }
    o += r->L;
  }
  const double t1 = now_ms();
  const double held = slot_held_bytes(sl, sl->V);
  std::lock_guard<std::mutex> lk(s->mu);
  // what the slot really holds now replaces the estimate charged for it
  s->used += held - sl->held;
  sl->held = held;
  sl->busy = false;
  for (Request* r : batch) {
    r->status = status;
    r->iters = iters;
    r->batch_cols = L;
    r->t_done = t1;
    r->done = true;
  }
  ++s->solves;
  s->columns += L;
  s->max_cols = std::max<long long>(s->max_cols, L);
  s->cv_done.notify_all();
}

void worker(mbicg_server* s, Slot* sl) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        s->cv_work.wait(lk, [&] {
          if (s->stop) return true;
          if (s->hold) return false;
          for (Request* r : s->pending)
            if (r->field == sl->field) return true;
          return false;
        });
        if (s->stop) return;
        bool no_memory = false;
        batch = take_batch(s, sl, &no_memory);
        if (!batch.empty()) break;
        if (!no_memory) {
          s->cv_done.wait(lk);
          continue;
        }
        // the oldest request does not fit: idle slots give their workspaces
        // back (their threads wait for the lock, so their contexts are not in
        // use), then, if that was not enough, wait for a running solve
        ++s->mem_waits;
        bool freed = false, running = false;
        for (Slot* o : s->slots) {
          running = running || o->busy;
          if (o != sl && !o->busy && o->held > 0) {
            release_slot_workspace(s, o);
            freed = true;
          }
        }
        if (freed) continue;
        if (running) {
          s->cv_done.wait(lk);
          continue;
        }
        // nothing runs and no idle slot holds memory, yet the oldest request
        // of this field does not fit: fields added after it was submitted
        // took the budget, and it can never be admitted.  It ends with
        // MBICG_ENOMEM.
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
          if ((*it)->field == sl->field) {
            Request* r = *it;
            s->pending.erase(it);
            r->X.assign(2 * (size_t)sl->V * 12 * r->L, 0.0);
            r->tres.assign(r->L, 0.0);
            r->status = MBICG_ENOMEM;
            r->t_start = r->t_done = now_ms();
            r->done = true;
            break;
          }
        s->cv_done.notify_all();
      }
      sl->busy = true;
    }
    run_batch(s, sl, batch);
    s->cv_work.notify_all();  // memory it gave back may admit another slot's block
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

void free_slot(Slot* sl) {
  if (sl->dB) cudaFree(sl->dB);
  if (sl->dX) cudaFree(sl->dX);
  if (sl->dS) cudaFree(sl->dS);
  if (sl->ctx) mbicg_destroy(sl->ctx);
  delete sl;
}

}  // namespace

extern "C" {

int mbicg_server_create(mbicg_server** out, int device, double hbm_budget_gb) {
  if (!out || !(hbm_budget_gb > 0)) return MBICG_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MBICG_ECUDA;
  }
  mbicg_server* s = new mbicg_server();
  s->device = device;
  s->budget = hbm_budget_gb * 1e9;
  *out = s;
  return MBICG_OK;
}

int mbicg_server_add_field(mbicg_server* s, const int dims[4], const double* U, const mbicg_params* p, int max_slots,
                           int* field_id) {
  if (!s || !dims || !U || !p || !field_id || max_slots < 1) return MBICG_EINVAL;
  Field f;
  f.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    f.dims[mu] = dims[mu];
    f.V *= dims[mu];
  }
  f.params = *p;
  const double need = slot_fixed_bytes(f.V);
  std::vector<Slot*> made;
  int rc = MBICG_OK;
  // the new field's index is the list's length until this call appends it
  std::lock_guard<std::mutex> add_lk(s->add_mu);
  cudaSetDevice(s->device);
  for (int k = 0; k < max_slots; ++k) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->used + need > s->budget) break;  // admission by HBM footprint
    }
    Slot* sl = new Slot();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      sl->field = (int)s->fields.size();
    }
    sl->V = f.V;
    sl->params = f.params;
    if ((rc = mbicg_create(&sl->ctx, dims, s->device, nullptr)) != MBICG_OK ||
        (rc = mbicg_load_gauge(sl->ctx, U)) != MBICG_OK) {
      free_slot(sl);
      break;
    }
    // the links are resident; the staging buffer of their upload is not kept
    ctx_release_workspace(sl->ctx);
    made.push_back(sl);
    std::lock_guard<std::mutex> lk(s->mu);
    s->used += need;
  }
  if (made.empty()) return rc != MBICG_OK ? rc : MBICG_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  f.nslots = (int)made.size();
  s->fields.push_back(f);
  *field_id = (int)s->fields.size() - 1;
  for (Slot* sl : made) {
    s->slots.push_back(sl);
    sl->th = std::thread(worker, s, sl);
  }
  return MBICG_OK;
}

int mbicg_server_submit(mbicg_server* s, int field, const double* B, int L, double kappa, double tol,
                        long long* request_id) {
  if (!s || !B || !request_id || L < 1 || L > SERVE_MAXL || !(tol > 0)) return MBICG_EINVAL;
  if (on_device(B)) return MBICG_EINVAL;  // B is read on the host
  long long V = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (field < 0 || field >= (int)s->fields.size()) return MBICG_EINVAL;
    const Field& f = s->fields[field];
    // a block of this request alone must fit beside the slots' links
    double fixed = 0;
    for (const Field& g : s->fields) fixed += g.nslots * slot_fixed_bytes(g.V);
    if (fixed + solve_bytes(f.V, L, f.params) > s->budget) return MBICG_ENOMEM;
    V = f.V;
  }
  // the copy of B is made without the lock: the slots' bookkeeping goes on meanwhile
  Request* r = new Request();
  r->B.assign(B, B + 2 * (size_t)V * 12 * L);
  r->field = field;
  r->L = L;
  r->kappa = kappa;
  r->tol = tol;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  s->requests[r->id] = r;
  s->pending.push_back(r);
  *request_id = r->id;
  s->cv_work.notify_all();
  return MBICG_OK;
}

int mbicg_server_wait(mbicg_server* s, long long request_id, double* X, int* iters, double* true_res,
                      mbicg_request_info* info) {
  if (!s || (X && on_device(X))) return MBICG_EINVAL;
  Request* r = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end() || it->second->claimed) return MBICG_EINVAL;
    r = it->second;
    r->claimed = true;
    s->cv_done.wait(lk, [&] { return r->done; });
    s->requests.erase(request_id);
  }
  if (X) std::copy(r->X.begin(), r->X.end(), X);
  if (iters) *iters = r->iters;
  if (true_res) std::copy(r->tres.begin(), r->tres.end(), true_res);
  if (info) {
    info->queue_ms = r->t_start - r->t_submit;
    info->latency_ms = r->t_done - r->t_submit;
    info->start_ms = r->t_start;
    info->done_ms = r->t_done;
    info->batch_columns = r->batch_cols;
  }
  const int st = r->status;
  delete r;
  return st;
}

int mbicg_server_hold(mbicg_server* s, int hold) {
  if (!s) return MBICG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->hold = hold != 0;
  }
  s->cv_work.notify_all();
  return MBICG_OK;
}

int mbicg_server_stats(mbicg_server* s, long long* solves, long long* columns, long long* max_columns,
                       int* slots) {
  if (!s) return MBICG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (solves) *solves = s->solves;
  if (columns) *columns = s->columns;
  if (max_columns) *max_columns = s->max_cols;
  if (slots) *slots = (int)s->slots.size();
  return MBICG_OK;
}

int mbicg_server_memory(mbicg_server* s, double* used_gb, double* budget_gb, long long* memory_waits) {
  if (!s) return MBICG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (used_gb) *used_gb = s->used / 1e9;
  if (budget_gb) *budget_gb = s->budget / 1e9;
  if (memory_waits) *memory_waits = s->mem_waits;
  return MBICG_OK;
}

void mbicg_server_destroy(mbicg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();  // a slot waiting for memory goes back to its stop test
  for (Slot* sl : s->slots)
    if (sl->th.joinable()) sl->th.join();
  cudaSetDevice(s->device);
  for (Slot* sl : s->slots) free_slot(sl);
  for (auto& kv : s->requests) delete kv.second;
  delete s;
}

}  // extern "C"
