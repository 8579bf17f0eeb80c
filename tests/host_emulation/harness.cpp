// Host emulation of the library's FP64 operator and SAP kernels: every kernel
// body runs once per emulated (block, thread) in order.  device_parts.inc is
// cut out of the CUDA sources by the test (kernels and device helpers, no
// launches).
#include "device_parts.inc"

#include <vector>

EmuDim blockIdx, threadIdx, blockDim, gridDim;
namespace mbicg {
namespace emu_dslash {
unsigned char smem_raw[1 << 16];
}
}  // namespace mbicg
using namespace mbicg;

static Geom make_geom(const int* dims, const int* block) {
  Geom g{};
  g.V = 1;
  g.nd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.d[mu] = dims[mu];
    g.V *= dims[mu];
    g.blk[mu] = block ? block[mu] : dims[mu];
    g.nb[mu] = g.d[mu] / g.blk[mu];
    g.nd *= g.nb[mu];
  }
  g.Vd = g.V / g.nd;
  g.su3 = 1;
  geom_init_divisors(g);
  return g;
}

// runs body(slot, rhs) for a grid of n (site or slot) x L threads, one site per CTA row
template <typename F>
static void grid(int n, int L, F body) {
  blockDim = {(unsigned)L, 1, 1};
  gridDim = {(unsigned)n, 1, 1};
  for (int b = 0; b < n; ++b)
    for (int r = 0; r < L; ++r) {
      blockIdx = {(unsigned)b, 0, 0};
      threadIdx = {(unsigned)r, 0, 0};
      body();
    }
}

using C = cx<double>;

extern "C" {
// the operator with the launch shape of the library: CTAs of S sites, walked
// in time slabs where the library uses them
void emu_dslash(const int* dims, const double* U, const double* in, double* out, int L, double kappa, int S,
                int order) {
  const Geom g = make_geom(dims, nullptr);
  const int slice = g.d[0] * g.d[1] * g.d[2];
  const bool slabs = order == 1 && slice % S == 0 && g.d[3] % 8 == 0;
  const int nblk = (g.V + S - 1) / S;
  blockDim = {(unsigned)L, (unsigned)S, 1};
  gridDim = {(unsigned)nblk, 1, 1};
  for (int b = 0; b < nblk; ++b)
    for (int y = 0; y < S; ++y)
      for (int r = 0; r < L; ++r) {
        blockIdx = {(unsigned)b, 0, 0};
        threadIdx = {(unsigned)r, (unsigned)y, 0};
        emu_dslash::k_dslash_full<double>(g, (const C*)U, (const C*)in, (C*)out, L, kappa, slabs ? slice / S : 0,
                                          slabs ? 8 : 1);
      }
}
int emu_segment_of(int b, int wslice, int tt) { return emu_dslash::segment_of(b, wslice, tt); }
int emu_nslot(const int* dims, const int* block) {
  const Geom g = make_geom(dims, block);
  return (g.nd / 2) * g.Vd;
}
void emu_slot(const int* dims, const int* block, int colour, int slot, int* site, int* k) {
  const Geom g = make_geom(dims, block);
  int c[4], lc[4];
  colour_slot_coords(g, colour, slot, c, lc, k);
  *site = site_index(g, c);
}
void emu_sap_residual(const int* dims, const int* block, const double* U, int colour, const double* eta,
                      const double* psi, double* r, int L, double kappa, int psi_zero) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    emu_dslash::k_sap_residual<double>(g, colour, (const C*)U, (const C*)eta, (const C*)psi, (C*)r, L, kappa,
                                       psi_zero);
  });
}
void emu_sap_domain_apply(const int* dims, const int* block, const double* U, int colour, const double* r,
                          double* q, int L, double kappa) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    emu_dslash::k_sap_domain_apply<double>(g, colour, (const C*)U, (const C*)r, (C*)q, nullptr, L, kappa, 1);
  });
}
// ABI blocks -> FP16 storage -> the FP16 operator -> ABI, with the link rows
// rounded to FP16 as the library stores them
void emu_half_operator(const int* dims, const double* U, const double* in, double* out, int L, double kappa) {
  const Geom g = make_geom(dims, nullptr);
  const long long V = g.V;
  std::vector<__half2> l16((size_t)V * 24), q((size_t)V * L * 12), qo((size_t)V * L * 12);
  std::vector<float> sc((size_t)V * L), so((size_t)V * L);
  grid(1, 1, [&] { emu_half::k_links_to_half(V * 4, (const C*)U, l16.data()); });  // grid-stride
  blockDim = {256, 1, 1};
  for (long long idx = 0; idx < V * L; ++idx) {
    blockIdx = {(unsigned)(idx / 256), 0, 0};
    threadIdx = {(unsigned)(idx % 256), 0, 0};
    emu_half::k_abi_to_half(V, L, (const C*)in, q.data(), sc.data());
  }
  grid(g.V, L, [&] {
    emu_half::k_dslash_half(g, l16.data(), q.data(), sc.data(), qo.data(), so.data(), L, (float)kappa);
  });
  blockDim = {256, 1, 1};
  for (long long idx = 0; idx < V * L; ++idx) {
    blockIdx = {(unsigned)(idx / 256), 0, 0};
    threadIdx = {(unsigned)(idx % 256), 0, 0};
    emu_half::k_half_to_abi(V, L, qo.data(), so.data(), (C*)out);
  }
}
void emu_mr_update(const int* dims, const int* block, int colour, const double* omega, double* r, const double* q,
                   double* x, double* psi, int L, int first, int last) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    emu_sap::k_mr_update<double>(g, colour, omega, (C*)r, (const C*)q, (C*)x, (C*)psi, L, first, last);
  });
}
}
