// Host emulation of the library's FP64 operator, SAP and clover kernels: every kernel
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
// in time slabs where the library uses them; cm: 0 Wilson, 1 Jacobi-
// preconditioned clover (clov = T^{-1}), 2 clover (clov = C)
void emu_dslash(const int* dims, const double* U, const double* in, double* out, int L, double kappa,
                const double* clov, int cm, int S, int order) {
  const Geom g = make_geom(dims, nullptr);
  const int slice = g.d[0] * g.d[1] * g.d[2];
  const bool slabs = order == 1 && slice % S == 0 && g.d[3] % 8 == 0;
  const int ws = slabs ? slice / S : 0, tt = slabs ? 8 : 1;
  const int nblk = (g.V + S - 1) / S;
  blockDim = {(unsigned)L, (unsigned)S, 1};
  gridDim = {(unsigned)nblk, 1, 1};
  for (int b = 0; b < nblk; ++b)
    for (int y = 0; y < S; ++y)
      for (int r = 0; r < L; ++r) {
        blockIdx = {(unsigned)b, 0, 0};
        threadIdx = {(unsigned)r, (unsigned)y, 0};
        if (cm == 1)
          emu_dslash::k_dslash_full<double, 1>(g, (const C*)U, (const C*)in, (C*)out, L, kappa, clov, ws, tt);
        else if (cm == 2)
          emu_dslash::k_dslash_full<double, 2>(g, (const C*)U, (const C*)in, (C*)out, L, kappa, clov, ws, tt);
        else
          emu_dslash::k_dslash_full<double, 0>(g, (const C*)U, (const C*)in, (C*)out, L, kappa, nullptr, ws, tt);
      }
}
void emu_clover_field(const int* dims, const double* U, double csw, double* Cl) {
  const Geom g = make_geom(dims, nullptr);
  grid(1, 1, [&] { emu_clover::k_clover_field(g, (const C*)U, csw, Cl); });  // grid-stride loop over sites
}
int emu_clover_terms(long long nsite, const double* Cl, double kappa, double* Ti64, float* Ti32, float* C32) {
  int status = 0;
  grid(1, 1, [&] { emu_clover::k_clover_terms(2 * nsite, Cl, kappa, Ti64, Ti32, C32, &status); });
  return status;
}
void emu_clover_abi(long long nsite, int L, const double* M, const double* in, double* out) {
  blockDim = {256, 1, 1};
  for (long long idx = 0; idx < nsite * L; ++idx) {
    blockIdx = {(unsigned)(idx / 256), 0, 0};
    threadIdx = {(unsigned)(idx % 256), 0, 0};
    emu_clover::k_clover_abi(nsite, L, M, (const C*)in, (C*)out);
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
                      const double* psi, double* r, int L, double kappa, int psi_zero, const double* tinv) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    if (tinv)
      emu_dslash::k_sap_residual<double, 1>(g, colour, (const C*)U, (const C*)eta, (const C*)psi, (C*)r, L, 0, kappa,
                                            psi_zero, tinv);
    else
      emu_dslash::k_sap_residual<double, 0>(g, colour, (const C*)U, (const C*)eta, (const C*)psi, (C*)r, L, 0, kappa,
                                            psi_zero, nullptr);
  });
}
void emu_sap_domain_apply(const int* dims, const int* block, const double* U, int colour, const double* r,
                          double* q, int L, double kappa, const double* tinv) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    if (tinv)
      emu_dslash::k_sap_domain_apply<double, 1>(g, colour, (const C*)U, (const C*)r, (C*)q, nullptr, L, kappa, 1,
                                                tinv);
    else
      emu_dslash::k_sap_domain_apply<double, 0>(g, colour, (const C*)U, (const C*)r, (C*)q, nullptr, L, kappa, 1,
                                                nullptr);
  });
}
void emu_ssor_level(const int* dims, const int* block, const double* U, const double* tinv, int colour,
                    const double* y, double* z, int L, double komega, const int* local, int count, int fwd) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * count, L, [&] {
    const C* U_ = (const C*)U;
    if (tinv) {
      if (fwd) emu_dslash::k_ssor_level<double, 1, true>(g, colour, U_, tinv, (const C*)y, (C*)z, L, komega, local, count);
      else emu_dslash::k_ssor_level<double, 1, false>(g, colour, U_, tinv, (const C*)y, (C*)z, L, komega, local, count);
    } else {
      if (fwd) emu_dslash::k_ssor_level<double, 0, true>(g, colour, U_, nullptr, (const C*)y, (C*)z, L, komega, local, count);
      else emu_dslash::k_ssor_level<double, 0, false>(g, colour, U_, nullptr, (const C*)y, (C*)z, L, komega, local, count);
    }
  });
}
void emu_ssor_combine(const int* dims, const int* block, int colour, const double* pv, const double* qv,
                      const double* pqv, double* term, double* acc, int L, double omega) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] {
    emu_sap::k_ssor_combine<double>(g, colour, (const C*)pv, (const C*)qv, (const C*)pqv, (C*)term, (C*)acc, L, omega);
  });
}
void emu_colour_add(const int* dims, const int* block, int colour, const double* x, double* psi, int L) {
  const Geom g = make_geom(dims, block);
  grid((g.nd / 2) * g.Vd, L, [&] { emu_sap::k_colour_add<double>(g, colour, (const C*)x, (C*)psi, L); });
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
