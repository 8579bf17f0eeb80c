// Host emulation of the library's FP64 operator and SAP kernels: every kernel
// body runs once per emulated (block, thread) in order.  device_parts.inc is
// cut out of the CUDA sources by the test (kernels and device helpers, no
// launches).
#include "device_parts.inc"

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
void emu_dslash(const int* dims, const double* U, const double* in, double* out, int L, double kappa) {
  const Geom g = make_geom(dims, nullptr);
  grid(g.V, L, [&] { emu_dslash::k_dslash_full<double>(g, (const C*)U, (const C*)in, (C*)out, L, kappa); });
}
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
void emu_mr_update(const int* dims, const int* block, int colour, const double* omega, double* r, const double* q,
                   double* x, double* psi, int L, int first, int last) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    emu_sap::k_mr_update<double>(g, colour, omega, (C*)r, (const C*)q, (C*)x, (C*)psi, L, first, last);
  });
}
}
