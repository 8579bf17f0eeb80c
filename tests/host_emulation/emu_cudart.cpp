// The CUDA runtime calls of the library's host code, over host memory, for
// the emulated build: allocations are malloc'd and recorded (so the
// library's host/device pointer test sees its own buffers as device memory),
// copies and fills are immediate, streams are tokens, an event records the
// host clock (launches run to completion when they are made, so the time
// between two events is the emulated work between them), and stream capture
// is refused (the solver then runs its iterations eagerly).
#include <cuda_runtime.h>

#include <chrono>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "shim_threads.h"

thread_local EmuThread emu_t;
EmuDim blockDim, gridDim;
int emu_bad_access = 0;

namespace {
std::mutex mu;
std::map<const char*, size_t> device_allocs, host_allocs;
std::map<const char*, int> owners;  // device allocations of a device other than 0
int owner_of(const void* p) {
  std::lock_guard<std::mutex> g(mu);
  auto it = owners.find(static_cast<const char*>(p));
  return it == owners.end() ? 0 : it->second;
}
int kind_of(const void* p) {  // 2 device, 1 pinned host, 0 other
  std::lock_guard<std::mutex> g(mu);
  const char* c = static_cast<const char*>(p);
  for (auto* m : {&device_allocs, &host_allocs}) {
    auto it = m->upper_bound(c);
    if (it != m->begin()) {
      --it;
      if (c < it->first + it->second) return m == &device_allocs ? 2 : 1;
    }
  }
  return 0;
}
void* alloc(size_t n, std::map<const char*, size_t>& m) {
#if defined(__SANITIZE_ADDRESS__)
  // exactly n bytes, so that the sanitizer reports any access past the end
  void* p = nullptr;
  if (posix_memalign(&p, 256, n ? n : 1) != 0) return nullptr;
#else
  void* p = aligned_alloc(256, ((n + 255) / 256) * 256 + 256);
  if (!p) return nullptr;
#endif
  memset(p, 0xff, n);  // device memory starts with no particular content: NaN bytes
  std::lock_guard<std::mutex> g(mu);
  m[static_cast<const char*>(p)] = n;
  return p;
}
void release(void* p, std::map<const char*, size_t>& m) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> g(mu);
    m.erase(static_cast<const char*>(p));
    owners.erase(static_cast<const char*>(p));
  }
  free(p);
}
int token = 1;
std::map<size_t, std::chrono::steady_clock::time_point> event_times;
}  // namespace

extern "C" {
cudaError_t cudaMalloc(void** p, size_t n) {
  *p = alloc(n, device_allocs);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void* p) {
  release(p, device_allocs);
  return cudaSuccess;
}
cudaError_t cudaMallocHost(void** p, size_t n) {
  *p = alloc(n, host_allocs);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaHostAlloc(void** p, size_t n, unsigned int) {
  *p = alloc(n, host_allocs);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFreeHost(void* p) {
  release(p, host_allocs);
  return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, enum cudaMemcpyKind, cudaStream_t) {
  memmove(d, s, n);
  return cudaSuccess;
}
cudaError_t cudaMemcpy(void* d, const void* s, size_t n, enum cudaMemcpyKind) {
  memmove(d, s, n);
  return cudaSuccess;
}
cudaError_t cudaMemset(void* p, int v, size_t n) {
  memset(p, v, n);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t) {
  memset(p, v, n);
  return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaDeviceSynchronize(void) { return cudaSuccess; }
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int* d) {
  *d = 0;
  return cudaSuccess;
}
// a __device__ variable is a host variable here: its address is the "device" address
cudaError_t cudaGetSymbolAddress(void** p, const void* symbol) {
  *p = const_cast<void*>(symbol);
  return cudaSuccess;
}
cudaError_t cudaGetDeviceCount(int* n) {
  *n = 1;
  return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned int) {
  *s = reinterpret_cast<cudaStream_t>(static_cast<size_t>(++token));
  return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaPointerGetAttributes(struct cudaPointerAttributes* a, const void* p) {
  memset(a, 0, sizeof(*a));
  const int k = kind_of(p);
  a->type = k == 2 ? cudaMemoryTypeDevice : k == 1 ? cudaMemoryTypeHost : cudaMemoryTypeUnregistered;
  // unified addressing: registered host memory is mapped at its own address
  a->devicePointer = k >= 1 ? const_cast<void*>(p) : nullptr;
  a->hostPointer = k != 2 ? const_cast<void*>(p) : nullptr;
  a->device = k == 2 ? owner_of(p) : 0;
  return cudaSuccess;
}
// Test hook (no CUDA counterpart): the emulated device allocation at p is
// reported as memory of `device`.
void emu_set_owner(const void* p, int device) {
  std::lock_guard<std::mutex> g(mu);
  owners[static_cast<const char*>(p)] = device;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaPeekAtLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t e) { return e == cudaSuccess ? "no error" : "emulated runtime error"; }
cudaError_t cudaEventCreate(cudaEvent_t* e) {
  *e = reinterpret_cast<cudaEvent_t>(static_cast<size_t>(++token));
  return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t) {
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> g(mu);
  event_times[reinterpret_cast<size_t>(e)] = now;
  return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned int) { return cudaEventCreate(e); }
// launches run to completion when they are made, so stream order holds already
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t a, cudaEvent_t b) {
  std::lock_guard<std::mutex> g(mu);
  auto ia = event_times.find(reinterpret_cast<size_t>(a)), ib = event_times.find(reinterpret_cast<size_t>(b));
  if (ia == event_times.end() || ib == event_times.end()) return cudaErrorInvalidResourceHandle;
  *ms = std::chrono::duration<float, std::milli>(ib->second - ia->second).count();
  return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t e) {
  std::lock_guard<std::mutex> g(mu);
  event_times.erase(reinterpret_cast<size_t>(e));
  return cudaSuccess;
}
cudaError_t cudaStreamIsCapturing(cudaStream_t, enum cudaStreamCaptureStatus* st) {
  *st = cudaStreamCaptureStatusNone;  // capture is never begun
  return cudaSuccess;
}
cudaError_t cudaStreamBeginCapture(cudaStream_t, enum cudaStreamCaptureMode) { return cudaErrorNotSupported; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t* g) {
  *g = nullptr;
  return cudaErrorNotSupported;
}
cudaError_t cudaGraphInstantiate(cudaGraphExec_t*, cudaGraph_t, unsigned long long) { return cudaErrorNotSupported; }
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
// the device loop's conditional graph is refused too, so the solver falls back
// to one host check per eager iteration
cudaError_t cudaGraphCreate(cudaGraph_t*, unsigned int) { return cudaErrorNotSupported; }
cudaError_t cudaGraphConditionalHandleCreate(cudaGraphConditionalHandle*, cudaGraph_t, unsigned int, unsigned int) {
  return cudaErrorNotSupported;
}
cudaError_t cudaGraphAddNode(cudaGraphNode_t*, cudaGraph_t, const cudaGraphNode_t*, const cudaGraphEdgeData*, size_t,
                             struct cudaGraphNodeParams*) {
  return cudaErrorNotSupported;
}
cudaError_t cudaStreamBeginCaptureToGraph(cudaStream_t, cudaGraph_t, const cudaGraphNode_t*, const cudaGraphEdgeData*,
                                          size_t, enum cudaStreamCaptureMode) {
  return cudaErrorNotSupported;
}
cudaError_t cudaFuncSetAttribute(const void*, enum cudaFuncAttribute, int) { return cudaSuccess; }
cudaError_t cudaOccupancyMaxActiveClusters(int* n, const void*, const cudaLaunchConfig_t*) {
  *n = 3;
  return cudaSuccess;
}
}
