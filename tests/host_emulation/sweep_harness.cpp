// Threaded host emulation of the fused SAP sweep kernel (FP32): one host
// thread per CUDA thread, the clusters of a launch one after another.
// sweep_parts.inc is cut out of the CUDA sources by the test, with the inline
// PTX helpers (cluster window loads, 256-bit spinor loads) replaced by plain
// C++ and the shared-memory declarations bound to the emulated CTA arenas.
#include "sweep_parts.inc"

thread_local EmuThread emu_t;
EmuDim blockDim, gridDim;
int emu_bad_access = 0;
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

template <int DX, int DY, int DZ, int DT, int CX, int CY, int CZ, int CT, int NCOL>
static void run(const Geom& g, int colour, const float* links, const float* eta, float* psi, int L, float kappa,
                int psi_mode, int nmr, int mode, const double* table, int nclusters, const float* tinv) {
  using SH = emu_dslash::SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>;
  using C = cx<float>;
  emu_launch(nclusters, SH::CS, SH::NS, SH::smem_bytes(), [&] {
    if (tinv)
      emu_dslash::k_sap_sweep<DX, DY, DZ, DT, CX, CY, CZ, CT, 1, false, NCOL>(
          g, colour, (const C*)links, eta, nullptr, psi, nullptr, L, 0, L, kappa, psi_mode, nmr, mode, table, tinv);
    else
      emu_dslash::k_sap_sweep<DX, DY, DZ, DT, CX, CY, CZ, CT, 0, false, NCOL>(
          g, colour, (const C*)links, eta, nullptr, psi, nullptr, L, 0, L, kappa, psi_mode, nmr, mode, table, nullptr);
  });
}

// shape (8^4 domains): 0 clusters of 8 CTAs, one column per thread; 1
// clusters of 16 CTAs, two columns per thread; 2 clusters of 16 CTAs, one
// column per thread
extern "C" int emu_sweep(const int* dims, const int* block, int colour, const float* links, const float* eta,
                         float* psi, int L, float kappa, int psi_mode, int nmr, int mode, const double* table,
                         int nclusters, const float* tinv, int shape) {
  const Geom g = make_geom(dims, block);
  emu_bad_access = 0;
  const bool b8 = block[0] == 8 && block[1] == 8 && block[2] == 8 && block[3] == 8;
  const bool b4 = block[0] == 4 && block[1] == 4 && block[2] == 4 && block[3] == 4;
  if (b8 && shape == 1)
    run<8, 8, 8, 8, 1, 2, 2, 4, 2>(g, colour, links, eta, psi, L, kappa, psi_mode, nmr, mode, table, nclusters, tinv);
  else if (b8 && shape == 2)
    run<8, 8, 8, 8, 1, 2, 2, 4, 1>(g, colour, links, eta, psi, L, kappa, psi_mode, nmr, mode, table, nclusters, tinv);
  else if (b8)
    run<8, 8, 8, 8, 1, 2, 2, 2, 1>(g, colour, links, eta, psi, L, kappa, psi_mode, nmr, mode, table, nclusters, tinv);
  else if (b4)
    run<4, 4, 4, 4, 1, 1, 1, 1, 1>(g, colour, links, eta, psi, L, kappa, psi_mode, nmr, mode, table, nclusters, tinv);
  else return -1;
  return emu_bad_access ? -2 : 0;  // -2: an access left the cluster or a shared-memory arena
}
