// sap.cu — the SAP preconditioner of Sec. 2.2 (Schwarz alternating procedure,
// Luescher) on checkerboard-coloured domains:
//   psi = K sum_{j=0}^{ncycle-1} (1 - A K)^j eta,
//   K = [[B_EE, 0], [-B_OO A_OE B_EE, B_OO]],
// i.e. ncycle multiplicative cycles, each an E sweep then an O sweep on the
// updated residual.  The domain solves B_EE, B_OO are nmr minimal-residual
// steps started from zero, or the paper's SSOR solves (the wavefront kernels
// below).
//
// Each colour sweep recomputes the residual on that colour from eta and the
// current psi (r = eta - A psi), so no residual array has to be carried
// between sweeps, then runs the MR steps on all domains of the colour at once:
//   q = A_dom r (Dirichlet), omega = (q^H r)/(q^H q), x += omega r, r -= omega q
// and finally adds x to psi.  In FP32 (or FP16 storage), with 8^4 or 4^4
// domains of an SU(3) field and per-column or replayed frozen step lengths,
// the MR steps of a colour run on chip in one fused cluster kernel
// (dslash.cu).  Otherwise, per MR step: the domain
// operator with fused per-CTA dot products, a small kernel that forms the step
// lengths (per column, shared by the block, or read from a frozen table), and
// the update.  Frozen step lengths are recorded on this multi-kernel path.
#include <math.h>
#include <stdlib.h>

#include <type_traits>
#include <vector>

#include "internal.h"

namespace mbicg {

namespace {

// Step lengths omega[k][rhs] for the domains of one colour.
//   mode 0: per column; mode 1: shared by the columns (sums over them);
//   mode 2: frozen, recording: a NaN table entry is recorded from the mode-1
//           sums when the domain's residual is nonzero (otherwise omega
//           multiplies zero and *unset is raised); mode 3: frozen, replay.
__global__ void k_omega(int ndc, int nchunk, int L, int mode, const double* __restrict__ dots,
                        double* __restrict__ omega, double* __restrict__ table, int* __restrict__ unset) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ndc) return;
  if (mode == 0) {
    for (int rhs = 0; rhs < L; ++rhs) {
      double nre = 0, nim = 0, den = 0;
      for (int ch = 0; ch < nchunk; ++ch) {
        const double* d = dots + (((long long)k * nchunk + ch) * L + rhs) * 3;
        nre += d[0];
        nim += d[1];
        den += d[2];
      }
      omega[(k * L + rhs) * 2 + 0] = den > 0 ? nre / den : 0.0;
      omega[(k * L + rhs) * 2 + 1] = den > 0 ? nim / den : 0.0;
    }
    return;
  }
  double ore, oim;
  if (mode == 3 || (mode == 2 && !isnan(table[2 * k]))) {
    ore = table[2 * k];
    oim = table[2 * k + 1];
  } else {
    double nre = 0, nim = 0, den = 0;
    for (int rhs = 0; rhs < L; ++rhs)
      for (int ch = 0; ch < nchunk; ++ch) {
        const double* d = dots + (((long long)k * nchunk + ch) * L + rhs) * 3;
        nre += d[0];
        nim += d[1];
        den += d[2];
      }
    ore = den > 0 ? nre / den : 0.0;
    oim = den > 0 ? nim / den : 0.0;
    if (mode == 2) {
      if (den > 0) {
        table[2 * k] = ore;
        table[2 * k + 1] = oim;
      } else {
        atomicOr(unset, 1);
      }
    }
  }
  for (int rhs = 0; rhs < L; ++rhs) {
    omega[(k * L + rhs) * 2 + 0] = ore;
    omega[(k * L + rhs) * 2 + 1] = oim;
  }
}

// x (+)= omega r; last step: psi += x, otherwise r -= omega q
template <typename R>
__global__ void __launch_bounds__(512) k_mr_update(Geom g, int colour, const double* __restrict__ omega,
                                                   cx<R>* __restrict__ r, const cx<R>* __restrict__ q,
                                                   cx<R>* __restrict__ x, cx<R>* __restrict__ psi, int L,
                                                   int first, int last) {
  const int rhs = threadIdx.x;
  const int slot = blockIdx.x * blockDim.y + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const int s = site_index(g, c);
  const size_t off = (size_t)(s * L + rhs) * 12;
  const cx<R> om = mk((R)omega[(k * L + rhs) * 2], (R)omega[(k * L + rhs) * 2 + 1]);
  Spinor<R> rv, xv;
  load_spinor(r + off, rv);
  if (first) zero(xv);
  else load_spinor(x + off, xv);
#pragma unroll
  for (int j = 0; j < 12; ++j) cmac((&xv.c[0][0])[j], om, (&rv.c[0][0])[j]);
  if (last) {
    Spinor<R> pv;
    load_spinor(psi + off, pv);
#pragma unroll
    for (int j = 0; j < 12; ++j) (&pv.c[0][0])[j] = (&pv.c[0][0])[j] + (&xv.c[0][0])[j];
    store_spinor(psi + off, pv);
  } else {
    Spinor<R> qv;
    load_spinor(q + off, qv);
    const cx<R> mom = mk(-om.re, -om.im);
#pragma unroll
    for (int j = 0; j < 12; ++j) cmac((&rv.c[0][0])[j], mom, (&qv.c[0][0])[j]);
    store_spinor(x + off, xv);
    store_spinor(r + off, rv);
  }
}

// SSOR: term -= Ahat term with Ahat term = (pv + qv + (omega - 2) pqv) / omega,
// then acc += term, on the sites of one colour
template <typename R>
__global__ void __launch_bounds__(512) k_ssor_combine(Geom g, int colour, const cx<R>* __restrict__ pv,
                                                      const cx<R>* __restrict__ qv, const cx<R>* __restrict__ pqv,
                                                      cx<R>* __restrict__ term, cx<R>* __restrict__ acc, int L,
                                                      double omega) {
  const int rhs = threadIdx.x;
  const int slot = blockIdx.x * blockDim.y + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const size_t off = (size_t)(site_index(g, c) * L + rhs) * 12;
  const R inv = (R)(1.0 / omega), w2 = (R)(omega - 2.0);
  Spinor<R> a, b, e, t, s;
  load_spinor(pv + off, a);
  load_spinor(qv + off, b);
  load_spinor(pqv + off, e);
  load_spinor(term + off, t);
  load_spinor(acc + off, s);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const cx<R> ah = inv * ((&a.c[0][0])[j] + (&b.c[0][0])[j] + w2 * (&e.c[0][0])[j]);
    cx<R>& tj = (&t.c[0][0])[j];
    tj = tj - ah;
    (&s.c[0][0])[j] = (&s.c[0][0])[j] + tj;
  }
  store_spinor(term + off, t);
  store_spinor(acc + off, s);
}

// psi += x on the sites of one colour
template <typename R>
__global__ void __launch_bounds__(512) k_colour_add(Geom g, int colour, const cx<R>* __restrict__ x,
                                                    cx<R>* __restrict__ psi, int L) {
  const int rhs = threadIdx.x;
  const int slot = blockIdx.x * blockDim.y + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const size_t off = (size_t)(site_index(g, c) * L + rhs) * 12;
  Spinor<R> a, b;
  load_spinor(x + off, a);
  load_spinor(psi + off, b);
#pragma unroll
  for (int j = 0; j < 12; ++j) (&b.c[0][0])[j] = (&b.c[0][0])[j] + (&a.c[0][0])[j];
  store_spinor(psi + off, b);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side of the driver
// ---------------------------------------------------------------------------
namespace {


// out = B y on every domain of one colour (Sec. 2.2):
//   B = (1 - omega U)^{-1} [sum_{j=0}^{nssor} (1 - Ahat)^j] (1 - omega L)^{-1},
//   Ahat = (1/omega) [(1 - omega L)^{-1} + (1 - omega U)^{-1}
//                     + (omega - 2) (1 - omega L)^{-1} (1 - omega U)^{-1}],
// each triangular inverse a substitution over the wavefront levels (L: from
// the highest level down, U: from level 0 up).
template <typename R>
void ssor_solve(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const R* tinv, const cx<R>* y,
                cx<R>* out, int L, double kappa, const SsorParams& sp, SapWork& w) {
  cx<R>* acc = static_cast<cx<R>*>(w.ssor[0]);
  cx<R>* term = static_cast<cx<R>*>(w.ssor[1]);
  cx<R>* pv = static_cast<cx<R>*>(w.ssor[2]);
  cx<R>* pqv = static_cast<cx<R>*>(w.ssor[3]);
  cx<R>* qv = static_cast<cx<R>*>(w.q);
  const int nlev = (int)w.level_off.size() - 1;
  const double ko = kappa * sp.omega;
  auto substitute = [&](bool fwd, const cx<R>* src, cx<R>* dst) {
    for (int n = 0; n < nlev; ++n) {
      const int lev = fwd ? nlev - 1 - n : n;
      const int a = w.level_off[lev], b = w.level_off[lev + 1];
      ssor_level<R>(ex, g, colour, links, tinv, src, dst, L, ko, w.levels + a, b - a, fwd);
    }
  };
  const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
  const int nslot = (g.nd / 2) * g.Vd;
  substitute(true, y, acc);  // acc = (1 - omega L)^{-1} y
  cudaMemcpyAsync(term, acc, sizeof(cx<R>) * 12 * (size_t)g.V * L, cudaMemcpyDeviceToDevice, ex.stream);
  for (int j = 1; j <= sp.nssor; ++j) {
    substitute(false, term, qv);  // (1 - omega U)^{-1} term
    substitute(true, term, pv);   // (1 - omega L)^{-1} term
    substitute(true, qv, pqv);    // (1 - omega L)^{-1} (1 - omega U)^{-1} term
    k_ssor_combine<R><<<(unsigned)(nslot / S), dim3(L, S), 0, ex.stream>>>(g, colour, pv, qv, pqv, term, acc, L,
                                                                          sp.omega);
    ++*ex.launches;
  }
  substitute(false, acc, out);  // out = (1 - omega U)^{-1} acc
}

}  // namespace

cudaError_t sap_prepare_ssor(const Geom& g, SapWork& w, cudaStream_t stream) {
  const int* b = g.blk;
  const int nlev = (b[0] - 1) + (b[1] - 1) + (b[2] - 1) + (b[3] - 1) + 1;
  std::vector<std::vector<int>> by(nlev);
  for (int l = 0; l < g.Vd; ++l) {
    const int x = l % b[0], y = (l / b[0]) % b[1], z = (l / (b[0] * b[1])) % b[2], t = l / (b[0] * b[1] * b[2]);
    by[x + y + z + t].push_back(l);
  }
  w.level_host.clear();
  w.level_off.assign(1, 0);
  for (const auto& v : by) {
    w.level_host.insert(w.level_host.end(), v.begin(), v.end());
    w.level_off.push_back((int)w.level_host.size());
  }
  return cudaMemcpyAsync(w.levels, w.level_host.data(), sizeof(int) * w.level_host.size(), cudaMemcpyHostToDevice,
                         stream);
}

template <typename R>
void sap_apply(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* eta, cx<R>* psi, int L,
               double kappa, int ncycle, int nmr, int mr_mode, double* table, int* unset, SapWork& w,
               const R* tinv, const SsorParams* ssor) {
  cx<R>* r = static_cast<cx<R>*>(w.r);
  cx<R>* q = static_cast<cx<R>*>(w.q);
  cx<R>* x = static_cast<cx<R>*>(w.x);
  const int ndc = g.nd / 2;
  const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
  const int nslot = ndc * g.Vd;
  cudaMemsetAsync(psi, 0, sizeof(cx<R>) * 12 * (size_t)g.V * L, ex.stream);
  if (ssor) {
    // K with SSOR domain solves: per colour, r = eta - A psi, x = B r, psi += x
    for (int cyc = 0; cyc < ncycle; ++cyc)
      for (int colour = 0; colour < 2; ++colour) {
        {
          Timed t(ex, KC_SAP_RESID);
          sap_residual<R>(ex, g, colour, links, eta, psi, r, L, kappa, cyc == 0 && colour == 0, tinv, 0, 0, w.links12);
        }
        Timed t(ex, KC_SAP_DOMAIN);
        ssor_solve<R>(ex, g, colour, links, tinv, r, x, L, kappa, *ssor, w);
        k_colour_add<R><<<(unsigned)(nslot / S), dim3(L, S), 0, ex.stream>>>(g, colour, x, psi, L);
        ++*ex.launches;
      }
    return;
  }
  const char* fused_env = getenv("MBICG_SAP_FUSED");
  const bool allow_fused = !(fused_env && fused_env[0] == '0');
  for (int cyc = 0; cyc < ncycle; ++cyc) {
    for (int colour = 0; colour < 2; ++colour) {
      if constexpr (std::is_same<R, float>::value) {
        if (allow_fused && sap_sweep_fusable(g, mr_mode)) {
          // the colour's residual eta - A psi by the streaming residual
          // kernel, then the MR steps on chip (psi = 0 before the first sweep:
          // the residual is eta itself)
          const double* tab = table ? table + ((long long)cyc * 2 + colour) * nmr * ndc * 2 : nullptr;
          const bool first = cyc == 0 && colour == 0;
          if (!first) {
            Timed t(ex, KC_SAP_RESID);
            sap_residual<R>(ex, g, colour, links, eta, psi, r, L, kappa, false, tinv, 0, 0, w.links12);
          }
          Timed t(ex, KC_SAP_SWEEP);
          sap_sweep_fused(ex, g, colour, links, first ? eta : r, psi, L, kappa, first ? 1 : 2, nmr, mr_mode, tab,
                          tinv);
          continue;
        }
      }
      {
        Timed t(ex, KC_SAP_RESID);
        sap_residual<R>(ex, g, colour, links, eta, psi, r, L, kappa, cyc == 0 && colour == 0, tinv, 0, 0, w.links12);
      }
      for (int it = 0; it < nmr; ++it) {
        const bool need_dots = (mr_mode != 3);
        int nchunk = g.Vd / S;
        // replaying frozen step lengths, the last step needs no A_dom r: only x + omega r
        if (need_dots || it < nmr - 1) {
          Timed t(ex, KC_SAP_DOMAIN);
          sap_domain_apply<R>(ex, g, colour, links, r, q, need_dots ? w.dots : nullptr, L, kappa, &nchunk, tinv);
        }
        Timed t(ex, KC_SAP_UPDATE);
        double* tab = table ? table + (((long long)cyc * 2 + colour) * nmr + it) * ndc * 2 : nullptr;
        k_omega<<<(ndc + 127) / 128, 128, 0, ex.stream>>>(ndc, nchunk, L, mr_mode, w.dots, w.omega, tab, unset);
        ++*ex.launches;
        k_mr_update<R><<<(unsigned)(nslot / S), dim3(L, S), 0, ex.stream>>>(
            g, colour, w.omega, r, q, x, psi, L, it == 0 ? 1 : 0, it == nmr - 1 ? 1 : 0);
        ++*ex.launches;
      }
    }
  }
}

void sap_apply_h(const Exec& ex, const Geom& g, const cx<float>* links, const SapHalf& h, int L, double kappa,
                 int ncycle, int nmr, int mr_mode, const double* table, const float* tinv) {
  const int ndc = g.nd / 2;
  const size_t nsp = (size_t)g.V * L;
  // psi = 0 (FP16 zeros and zero scales): the residual kernel reads psi on
  // every site from the second sweep on
  cudaMemsetAsync(h.psi, 0, sizeof(__half2) * 12 * nsp, ex.stream);
  cudaMemsetAsync(h.psi_sc, 0, sizeof(float) * nsp, ex.stream);
  for (int cyc = 0; cyc < ncycle; ++cyc)
    for (int colour = 0; colour < 2; ++colour) {
      const double* tab = table ? table + ((long long)cyc * 2 + colour) * nmr * ndc * 2 : nullptr;
      const bool first = cyc == 0 && colour == 0;
      if (!first) {
        Timed t(ex, KC_SAP_RESID);
        sap_residual_h(ex, g, colour, links, h.eta, h.eta_sc, h.psi, h.psi_sc, h.r, h.r_sc, L, kappa, tinv);
      }
      Timed t(ex, KC_SAP_SWEEP);
      sap_sweep_fused_h(ex, g, colour, links, first ? h.eta : h.r, first ? h.eta_sc : h.r_sc, h.psi, h.psi_sc, L,
                        kappa, first ? 1 : 2, nmr, mr_mode, tab, tinv);
    }
}

template void sap_apply<float>(const Exec&, const Geom&, const cx<float>*, const cx<float>*, cx<float>*, int,
                               double, int, int, int, double*, int*, SapWork&, const float*, const SsorParams*);
template void sap_apply<double>(const Exec&, const Geom&, const cx<double>*, const cx<double>*, cx<double>*,
                                int, double, int, int, int, double*, int*, SapWork&, const double*,
                                const SsorParams*);

}  // namespace mbicg
