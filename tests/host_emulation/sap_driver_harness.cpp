// The library's SAP driver (sap_apply, with the launchers and kernels it
// uses) compiled for the host and run on the threaded emulator: the host code
// is the library's own, its launches run the emulated kernels to completion.
// driver_parts.inc is cut out of the CUDA sources by the test.
#include "driver_parts.inc"

#include <cstring>
#include <vector>

thread_local EmuThread emu_t;
EmuDim blockDim, gridDim;
int emu_bad_access = 0;

// the CUDA runtime calls the driver makes, on the host
extern "C" cudaError_t cudaFuncSetAttribute(const void*, enum cudaFuncAttribute, int) { return cudaSuccess; }
extern "C" cudaError_t cudaOccupancyMaxActiveClusters(int* n, const void*, const cudaLaunchConfig_t*) {
  *n = 3;  // three clusters at once: the persistent clusters share the items unevenly
  return cudaSuccess;
}
extern "C" cudaError_t cudaGetLastError(void) { return cudaSuccess; }
// per-kernel timing stays off in the emulation; these only satisfy the linker
extern "C" cudaError_t cudaEventCreate(cudaEvent_t*) { return cudaErrorNotSupported; }
extern "C" cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaErrorNotSupported; }
extern "C" cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaErrorNotSupported; }
extern "C" cudaError_t cudaEventElapsedTime(float*, cudaEvent_t, cudaEvent_t) { return cudaErrorNotSupported; }
extern "C" cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
// launches run to completion when they are made, so stream order holds already
extern "C" cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
extern "C" cudaError_t cudaStreamIsCapturing(cudaStream_t, enum cudaStreamCaptureStatus* st) {
  *st = cudaStreamCaptureStatusNone;
  return cudaSuccess;
}
extern "C" cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, enum cudaMemcpyKind, cudaStream_t) {
  memmove(d, s, n);
  return cudaSuccess;
}
extern "C" cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t) {
  memset(p, v, n);
  return cudaSuccess;
}

using namespace mbicg;

static Geom make_geom(const int* dims, const int* block) {
  Geom g{};
  g.V = 1;
  g.nd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.d[mu] = dims[mu];
    g.V *= dims[mu];
    g.blk[mu] = block[mu];
    g.nb[mu] = g.d[mu] / g.blk[mu];
    g.nd *= g.nb[mu];
  }
  g.Vd = g.V / g.nd;
  g.su3 = 1;
  geom_init_divisors(g);
  return g;
}

template <typename R>
static int run(const int* dims, const int* block, const void* links, const void* eta, void* psi, int L, double kappa,
               int ncycle, int nmr, int mode, double* table, int* unset) {
  const Geom g = make_geom(dims, block);
  const size_t nl = (size_t)g.V * 12 * L;
  std::vector<cx<R>> r(nl), q(nl), x(nl);
  const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
  std::vector<double> dots((size_t)(g.nd / 2) * (g.Vd / S) * L * 3), omega((size_t)(g.nd / 2) * L * 2);
  SapWork w;
  w.r = r.data();
  w.q = q.data();
  w.x = x.data();
  w.dots = dots.data();
  w.omega = omega.data();
  long long launches = 0;
  Prof prof;  // off
  const Exec ex{nullptr, &launches, &prof};
  emu_bad_access = 0;
  sap_apply<R>(ex, g, (const cx<R>*)links, (const cx<R>*)eta, (cx<R>*)psi, L, kappa, ncycle, nmr, mode, table, unset,
               w);
  return emu_bad_access ? -1 : (int)launches;
}

extern "C" {
// psi = M_SAP eta; blocks in the internal layout, links [site][mu][3][3];
// returns the kernels launched (or -1 after an access outside a cluster)
int emu_sap_apply(int fp64, const int* dims, const int* block, const void* links, const void* eta, void* psi, int L,
                  double kappa, int ncycle, int nmr, int mode, double* table, int* unset) {
  return fp64 ? run<double>(dims, block, links, eta, psi, L, kappa, ncycle, nmr, mode, table, unset)
              : run<float>(dims, block, links, eta, psi, L, kappa, ncycle, nmr, mode, table, unset);
}
// lexicographic index of the k-th domain of a colour
int emu_colour_domain(const int* dims, const int* block, int colour, int k) {
  const Geom g = make_geom(dims, block);
  int b[4];
  colour_domain(g, colour, k, b);
  return b[0] + g.nb[0] * (b[1] + g.nb[1] * (b[2] + g.nb[2] * b[3]));
}
}
