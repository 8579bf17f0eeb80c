// noalloc.cu — an operator entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework's
// memory pool and must not grow device memory behind the pool's back,
// real-time or latency-bound loops that may not take the allocator's locks or
// wait for it, and programs whose device memory is fixed when they start.
// mbicg_apply_D_noalloc serves them: it computes the same FP32 Wilson-Dirac
// operator as mbicg_apply_D(..., MBICG_FP32) with the caller's device buffers
// and a fixed scratch area that is a file-scope __device__ array, so it needs
// no context, no cudaMalloc and no cudaFree.
//
// The scratch array exists once per device in every process that loads the
// library and is held until the process exits.  Every call shares it and it
// keeps the last call's contents; each region is written in full before it is
// read, so nothing needs clearing.  Two calls that overlap on the GPU (on two
// streams, or two host threads) race on the scratch and give wrong results.
// The host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so the address is fetched with
// cudaGetSymbolAddress, once per device with that device current, by the first
// call on that device; that first call should come before any stream capture
// begins on that device.
#include <mutex>

#include "../../include/mbicg.h"
#include "internal.h"

using namespace mbicg;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)MBICG_NOALLOC_SCRATCH_MB << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// p is device memory (or managed memory) of `device`: the kernels below
// dereference the caller's pointers directly, so memory of another device or
// of the host is refused.
bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // no error was pending on entry: this one is ours
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

// scratch bytes for V sites and L columns: FP32 links and two FP32 blocks
size_t scratch_bytes(long long V, int L) {
  const size_t links = round256(sizeof(cx<float>) * (size_t)V * 36);
  const size_t block = round256(sizeof(cx<float>) * (size_t)V * 12 * L);
  return links + 2 * block;
}

}  // namespace

extern "C" int mbicg_apply_D_noalloc(const int dims[4], const double* U, const double* in, double* out, int L,
                                     double kappa, void* cuda_stream) {
  if (!dims || !U || !in || !out || in == out) return MBICG_EINVAL;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || dims[mu] % 2 != 0 || dims[mu] > 4096) return MBICG_EINVAL;
    V *= dims[mu];
  }
  if (L < 1 || L > MAXL || V > (1ll << 27)) return MBICG_EINVAL;
  if (scratch_bytes(V, L) > NOALLOC_SCRATCH_BYTES) return MBICG_EINVAL;
  // an error left pending by earlier work of the caller is not this call's:
  // report it without launching (and without clearing it)
  if (cudaPeekAtLastError() != cudaSuccess) return MBICG_ECUDA;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= MAX_DEVICES) return MBICG_ECUDA;
  if (!on_device(U, device) || !on_device(in, device) || !on_device(out, device)) return MBICG_EINVAL;
  void* base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return MBICG_ECUDA;
  }
  // scratch: FP32 links, then the input and output blocks in the internal layout
  unsigned char* p = static_cast<unsigned char*>(base);
  cx<float>* U32 = reinterpret_cast<cx<float>*>(p);
  p += round256(sizeof(cx<float>) * (size_t)V * 36);
  cx<float>* a = reinterpret_cast<cx<float>*>(p);
  p += round256(sizeof(cx<float>) * (size_t)V * 12 * L);
  cx<float>* b = reinterpret_cast<cx<float>*>(p);

  Geom g{};
  g.V = (int)V;
  g.nd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.d[mu] = dims[mu];
    g.blk[mu] = dims[mu];
    g.nb[mu] = 1;
  }
  g.Vd = g.V;
  geom_init_divisors(g);
  long long launches = 0;
  const Exec ex{static_cast<cudaStream_t>(cuda_stream), &launches, nullptr};
  // each launch checked by itself, so the status reflects this call's launches only
  convert_block<double, float>(ex, V * 36, reinterpret_cast<const cx<double>*>(U), U32);
  if (cudaGetLastError() != cudaSuccess) return MBICG_ECUDA;
  abi_to_internal<float>(ex, V, L, reinterpret_cast<const cx<double>*>(in), a);
  if (cudaGetLastError() != cudaSuccess) return MBICG_ECUDA;
  dslash_full<float>(ex, g, U32, a, b, L, kappa);
  if (cudaGetLastError() != cudaSuccess) return MBICG_ECUDA;
  internal_to_abi<float>(ex, V, L, b, reinterpret_cast<cx<double>*>(out));
  if (cudaGetLastError() != cudaSuccess) return MBICG_ECUDA;
  return MBICG_OK;
}
