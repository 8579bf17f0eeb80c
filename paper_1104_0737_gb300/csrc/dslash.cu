// dslash.cu — the block Wilson-Dirac operator of Sec. 2.1,
//   (A phi)_x = phi_x - kappa eta_x,
//   eta_x = sum_mu [(1 - gamma_mu) U_mu(x) phi_{x+mu} + (1 + gamma_mu) U_mu(x-mu)^dag phi_{x-mu}],
// for L columns at once (Eq. (bloclhoppingterm)), plus the two restrictions
// of it that the SAP sweeps of Sec. 2.2 need: the residual eta - A psi on the
// sites of one domain colour, and the domain operator A_dom with Dirichlet
// boundaries (hops that leave the domain dropped) with the per-domain MR dot
// products fused in.
//
// One thread per (site, rhs); the CTA is (L rhs) x (S sites) so a warp covers
// consecutive (site, rhs) pairs, i.e. contiguous memory in the site-major
// layout, and the L threads of one site read the same eight links (served by
// L1 after the first).  Each hop loads the neighbour's 12 complex numbers with
// vector loads, projects to a half spinor (6 complex), multiplies by the link
// and rebuilds the lower spin components: 1320 flops per site and column for
// eta, 48 more for phi - kappa eta.
#include <cooperative_groups.h>
#include <algorithm>
#include <type_traits>
#include <stdio.h>
#include <stdlib.h>

#include "internal.h"
#include "tune.h"

namespace mbicg {

namespace {

// CTA size cap: 384 threads for FP32 with two CTAs per SM (<= 80 registers,
// 24 warps), 256 for FP64, whose spinors and links take twice the registers.
template <typename R>
constexpr int max_cta() { return sizeof(R) == 4 ? 384 : 256; }
template <typename R>
constexpr int min_ctas() { return sizeof(R) == 4 ? 2 : 1; }

// R12: the links are stored as their first two rows (FP32 SU(3) fields)
template <int MU, int SIGN, bool R12 = false, typename R>
__device__ __forceinline__ void hop(Spinor<R>& acc, const cx<R>* psi_nb, const cx<R>* link, bool flip) {
  Spinor<R> p;
  load_spinor(psi_nb, p);
  cx<R> h[2][3];
  project<MU, SIGN>(p, h);
  Link<R> u;
  if constexpr (R12) load_link12(link, u);
  else load_link(link, u);
  cx<R> w[2][3];
  const R ph = flip ? R(-1) : R(1);
  link_times<(SIGN > 0)>(u, h, ph, w);
  reconstruct_add<MU, SIGN>(acc, w);
}

// Accumulates eta for site s (coordinates c, coordinates inside its domain lc).
// element offset of (site, rhs) in a site-major block
__device__ __forceinline__ size_t spinor_offset(int s, int L, int rhs) { return (size_t)(s * L + rhs) * 12; }

// complex numbers per stored link: 9, or 6 for the two-row form
template <bool R12>
__host__ __device__ constexpr int link_stride() { return R12 ? 6 : 9; }

template <typename R, bool DIRICHLET, int MU, bool R12 = false>
__device__ __forceinline__ void hops_mu(const Geom& g, const cx<R>* __restrict__ links,
                                        const cx<R>* __restrict__ in, int L, int rhs, int s,
                                        const int c[4], const int lc[4], int stride, Spinor<R>& acc) {
  const int dm = g.d[MU];
  // forward: (1 - gamma_mu) U_mu(x) phi_{x+mu}
  if (!DIRICHLET || lc[MU] != g.blk[MU] - 1) {
    const bool wrap = (c[MU] == dm - 1);
    const int sn = wrap ? s - (dm - 1) * stride : s + stride;
    hop<MU, -1, R12>(acc, in + spinor_offset(sn, L, rhs), links + (size_t)(s * 4 + MU) * link_stride<R12>(),
                     MU == 3 && wrap);
  }
  // backward: (1 + gamma_mu) U_mu(x - mu)^dagger phi_{x-mu}
  if (!DIRICHLET || lc[MU] != 0) {
    const bool wrap = (c[MU] == 0);
    const int sn = wrap ? s + (dm - 1) * stride : s - stride;
    hop<MU, +1, R12>(acc, in + spinor_offset(sn, L, rhs), links + (size_t)(sn * 4 + MU) * link_stride<R12>(),
                     MU == 3 && wrap);
  }
}

template <typename R, bool DIRICHLET, bool R12 = false>
__device__ __forceinline__ void hopping(const Geom& g, const cx<R>* __restrict__ links,
                                        const cx<R>* __restrict__ in, int L, int rhs, int s,
                                        const int c[4], const int lc[4], Spinor<R>& acc) {
  zero(acc);
  const int st1 = g.d[0];
  const int st2 = st1 * g.d[1];
  const int st3 = st2 * g.d[2];
  hops_mu<R, DIRICHLET, 0, R12>(g, links, in, L, rhs, s, c, lc, 1, acc);
  hops_mu<R, DIRICHLET, 1, R12>(g, links, in, L, rhs, s, c, lc, st1, acc);
  hops_mu<R, DIRICHLET, 2, R12>(g, links, in, L, rhs, s, c, lc, st2, acc);
  hops_mu<R, DIRICHLET, 3, R12>(g, links, in, L, rhs, s, c, lc, st3, acc);
}

// The order in which the CTAs of the operator walk the lattice.  A CTA takes a
// segment of S consecutive sites; the segments are taken in slabs of tt time
// slices with the time slice running fastest, so the CTAs that read a site as
// a t +- 1 neighbour run close in time to the one that reads it as its own
// site and the data is still in L2 (in lexicographic order they are a whole
// time slice, ~40 MB at 32^3 x 64, L = 12, apart).  wslice = segments per time
// slice; tt = 1 keeps the lexicographic order.
__host__ __device__ __forceinline__ int segment_of(int b, int wslice, int tt) {
  if (tt <= 1) return b;
  const int per_slab = wslice * tt;
  const int slab = b / per_slab, r = b - slab * per_slab;
  const int w = r / tt, dt = r - w * tt;
  return (slab * tt + dt) * wslice + w;
}

// Clover variants of the operator (clover.cu): CM = 0 the Wilson matrix,
// CM = 1 the Jacobi-preconditioned A = 1 - kappa M H with M = T^{-1},
// CM = 2 D_c = 1 + kappa M - kappa H with M = C (M packed per site).
template <typename R, int CM>
__device__ __forceinline__ void finish_site(const R* __restrict__ clov, int s, R kappa, const Spinor<R>& p,
                                            Spinor<R>& acc) {
  if (CM == 1) {
    Spinor<R> h;
    herm_apply<R>(clov + (size_t)s * HERM_PER_SITE, acc, h);
    acc = h;
  } else if (CM == 2) {
    Spinor<R> cp;
    herm_apply<R>(clov + (size_t)s * HERM_PER_SITE, p, cp);
#pragma unroll
    for (int k = 0; k < 12; ++k) (&acc.c[0][0])[k] = (&acc.c[0][0])[k] - (&cp.c[0][0])[k];
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<R>& o = (&acc.c[0][0])[k];
    const cx<R> v = (&p.c[0][0])[k];
    o = mk(fma(-kappa, o.re, v.re), fma(-kappa, o.im, v.im));
  }
}

template <typename R, int CM, bool R12 = false>
__global__ void __launch_bounds__(max_cta<R>(), min_ctas<R>()) k_dslash_full(Geom g, const cx<R>* __restrict__ links,
                                                     const cx<R>* __restrict__ in,
                                                     cx<R>* __restrict__ out, int L, R kappa,
                                                     const R* __restrict__ clov, int wslice, int tt) {
  const int rhs = threadIdx.x;
  const int s = segment_of(blockIdx.x, wslice, tt) * blockDim.y + threadIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  Spinor<R> acc;
  hopping<R, false, R12>(g, links, in, L, rhs, s, c, c, acc);
  Spinor<R> p;
  load_spinor(in + spinor_offset(s, L, rhs), p);
  finish_site<R, CM>(clov, s, kappa, p, acc);
  store_spinor(out + spinor_offset(s, L, rhs), acc);
}

template <typename R, int CM, bool R12 = false>
__global__ void __launch_bounds__(max_cta<R>(), min_ctas<R>()) k_sap_residual(Geom g, int colour,
                                                      const cx<R>* __restrict__ links,
                                                      const cx<R>* __restrict__ eta,
                                                      const cx<R>* __restrict__ psi,
                                                      cx<R>* __restrict__ r, int L, int c0, R kappa,
                                                      int psi_zero, const R* __restrict__ clov) {
  const int rhs = c0 + threadIdx.x;
  const int slot = blockIdx.x * blockDim.y + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const int s = site_index(g, c);
  Spinor<R> e;
  if (!psi_zero) {
    // the hop sum first: eta and psi of the site are loaded after it, so that
    // they hold no registers across the eight hops
    Spinor<R> acc, p;
    hopping<R, false, R12>(g, links, psi, L, rhs, s, c, c, acc);
    if (CM == 1) {  // A = 1 - kappa T^{-1} H
      Spinor<R> h;
      herm_apply<R>(clov + (size_t)s * HERM_PER_SITE, acc, h);
      acc = h;
    }
    load_spinor(eta + spinor_offset(s, L, rhs), e);
    load_spinor(psi + spinor_offset(s, L, rhs), p);
    // r = eta - (psi - kappa eta_hop) = eta - psi + kappa eta_hop
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      cx<R>& ej = (&e.c[0][0])[j];
      const cx<R> pj = (&p.c[0][0])[j], aj = (&acc.c[0][0])[j];
      ej = mk(fma(kappa, aj.re, ej.re - pj.re), fma(kappa, aj.im, ej.im - pj.im));
    }
  } else {
    load_spinor(eta + spinor_offset(s, L, rhs), e);
  }
  store_spinor(r + spinor_offset(s, L, rhs), e);
}

// The residual of the preconditioner's FP16 storage (Sec. 2.2, SAP in reduced
// precision): r = eta - A psi on the sites of one colour with eta, psi and r
// stored as FP16 spinors with a per-(site, column) scale, FP32 links and FP32
// arithmetic.
template <int MU, int SIGN>
__device__ __forceinline__ void hop_h32(Spinor<float>& acc, const __half2* __restrict__ q, const float* __restrict__ sc,
                                        size_t i, const cx<float>* __restrict__ link, bool flip) {
  Spinor<float> p;
  load_spinor_h(q + i * 12, __ldg(sc + i), p);
  cx<float> h[2][3];
  project<MU, SIGN>(p, h);
  Link<float> u;
  load_link(link, u);
  cx<float> w[2][3];
  link_times<(SIGN > 0)>(u, h, flip ? -1.0f : 1.0f, w);
  reconstruct_add<MU, SIGN>(acc, w);
}

template <int MU>
__device__ __forceinline__ void hops_h32(const Geom& g, const cx<float>* __restrict__ links,
                                         const __half2* __restrict__ q, const float* __restrict__ sc, int L, int rhs,
                                         int s, const int c[4], int stride, Spinor<float>& acc) {
  const int dm = g.d[MU];
  {
    const bool wrap = (c[MU] == dm - 1);
    const int sn = wrap ? s - (dm - 1) * stride : s + stride;
    hop_h32<MU, -1>(acc, q, sc, (size_t)sn * L + rhs, links + (size_t)(s * 4 + MU) * 9, MU == 3 && wrap);
  }
  {
    const bool wrap = (c[MU] == 0);
    const int sn = wrap ? s + (dm - 1) * stride : s - stride;
    hop_h32<MU, 1>(acc, q, sc, (size_t)sn * L + rhs, links + (size_t)(sn * 4 + MU) * 9, MU == 3 && wrap);
  }
}

template <int CM>
__global__ void __launch_bounds__(384, 2) k_sap_residual_h(Geom g, int colour, const cx<float>* __restrict__ links,
                                                           const __half2* __restrict__ eta, const float* __restrict__ esc,
                                                           const __half2* __restrict__ psi,
                                                           const float* __restrict__ psc, __half2* __restrict__ r,
                                                           float* __restrict__ rsc, int L, int c0, float kappa,
                                                           const float* __restrict__ clov) {
  const int rhs = c0 + threadIdx.x;
  const int slot = blockIdx.x * blockDim.y + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const int s = site_index(g, c);
  const size_t i = (size_t)s * L + rhs;
  Spinor<float> acc, e, p;
  zero(acc);
  const int st1 = g.d[0], st2 = st1 * g.d[1], st3 = st2 * g.d[2];
  hops_h32<0>(g, links, psi, psc, L, rhs, s, c, 1, acc);
  hops_h32<1>(g, links, psi, psc, L, rhs, s, c, st1, acc);
  hops_h32<2>(g, links, psi, psc, L, rhs, s, c, st2, acc);
  hops_h32<3>(g, links, psi, psc, L, rhs, s, c, st3, acc);
  if (CM == 1) {  // A = 1 - kappa T^{-1} H
    Spinor<float> h;
    herm_apply<float>(clov + (size_t)s * HERM_PER_SITE, acc, h);
    acc = h;
  }
  load_spinor_h(eta + i * 12, __ldg(esc + i), e);
  load_spinor_h(psi + i * 12, __ldg(psc + i), p);
  // r = eta - (psi - kappa eta_hop)
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    cx<float>& ej = (&e.c[0][0])[j];
    const cx<float> pj = (&p.c[0][0])[j], aj = (&acc.c[0][0])[j];
    ej = mk(fmaf(kappa, aj.re, ej.re - pj.re), fmaf(kappa, aj.im, ej.im - pj.im));
  }
  store_spinor_h(r + i * 12, rsc + i, e);
}

template <typename R, int CM>
__global__ void __launch_bounds__(max_cta<R>(), min_ctas<R>()) k_sap_domain_apply(Geom g, int colour,
                                                          const cx<R>* __restrict__ links,
                                                          const cx<R>* __restrict__ r,
                                                          cx<R>* __restrict__ q,
                                                          double* __restrict__ dots, int L, R kappa,
                                                          int nchunk, const R* __restrict__ clov) {
  extern __shared__ unsigned char smem_raw[];
  R* red = reinterpret_cast<R*>(smem_raw);  // [3][S][L]
  const int rhs = threadIdx.x;
  const int S = blockDim.y;
  const int slot = blockIdx.x * S + threadIdx.y;
  int c[4], lc[4], k;
  colour_slot_coords(g, colour, slot, c, lc, &k);
  const int s = site_index(g, c);
  Spinor<R> acc, p;
  hopping<R, true>(g, links, r, L, rhs, s, c, lc, acc);
  if (CM == 1) {  // A_dom = 1 - kappa T^{-1} H_dom
    Spinor<R> h;
    herm_apply<R>(clov + (size_t)s * HERM_PER_SITE, acc, h);
    acc = h;
  }
  load_spinor(r + spinor_offset(s, L, rhs), p);
  R nre = 0, nim = 0, den = 0;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    cx<R>& o = (&acc.c[0][0])[j];
    const cx<R> v = (&p.c[0][0])[j];
    o = mk(fma(-kappa, o.re, v.re), fma(-kappa, o.im, v.im));
    // q^H r and q^H q
    nre = fma(o.re, v.re, fma(o.im, v.im, nre));
    nim = fma(o.re, v.im, fma(-o.im, v.re, nim));
    den = fma(o.re, o.re, fma(o.im, o.im, den));
  }
  store_spinor(q + spinor_offset(s, L, rhs), acc);
  if (dots == nullptr) return;  // uniform over the grid
  const int t = threadIdx.y * L + rhs;
  const int n = S * L;
  red[t] = nre;
  red[n + t] = nim;
  red[2 * n + t] = den;
  __syncthreads();
  for (int h = S >> 1; h > 0; h >>= 1) {
    if (threadIdx.y < h) {
      const int u = (threadIdx.y + h) * L + rhs;
      red[t] += red[u];
      red[n + t] += red[n + u];
      red[2 * n + t] += red[2 * n + u];
    }
    __syncthreads();
  }
  if (threadIdx.y == 0) {
    const int chunk = blockIdx.x % nchunk;
    double* d = dots + (((long long)k * nchunk + chunk) * L + rhs) * 3;
    d[0] = red[rhs];
    d[1] = red[n + rhs];
    d[2] = red[2 * n + rhs];
  }
}

// ---------------------------------------------------------------------------
// SSOR domain solves (Sec. 2.2): one wavefront level of a triangular
// substitution on every domain of one colour.  With L the forward and U the
// backward hops inside a domain (times kappa T^{-1} for the clover matrix),
// z = (1 - omega L)^{-1} y sets z_x = y_x + omega kappa [T^{-1}] (forward hops
// of z)_x, and a forward hop raises the level lx + ly + lz + lt of the site by
// one: the sites of one level depend only on the level above (below for U),
// so each level is one launch over all domains of the colour.
// ---------------------------------------------------------------------------
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void hop_in_domain(const Geom& g, const cx<R>* __restrict__ links,
                                              const cx<R>* __restrict__ in, int L, int rhs, int s, const int lc[4],
                                              int stride, Spinor<R>& acc) {
  // no hop inside a domain crosses the lattice boundary (>= 2 domains per direction)
  if (FWD) {
    if (lc[MU] != g.blk[MU] - 1)
      hop<MU, -1>(acc, in + spinor_offset(s + stride, L, rhs), links + (size_t)(s * 4 + MU) * 9, false);
  } else {
    if (lc[MU] != 0)
      hop<MU, +1>(acc, in + spinor_offset(s - stride, L, rhs), links + (size_t)((s - stride) * 4 + MU) * 9, false);
  }
}

template <typename R, int CM, bool FWD>
__global__ void __launch_bounds__(max_cta<R>(), min_ctas<R>()) k_ssor_level(Geom g, int colour,
                                                    const cx<R>* __restrict__ links, const R* __restrict__ tinv,
                                                    const cx<R>* __restrict__ y, cx<R>* z, int L, R komega,
                                                    const int* __restrict__ local, int count) {
  const int rhs = threadIdx.x;
  const int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= (g.nd / 2) * count) return;
  const int k = i / count;
  const int slot = k * g.Vd + __ldg(local + (i - k * count));
  int c[4], lc[4], kk;
  colour_slot_coords(g, colour, slot, c, lc, &kk);
  const int s = site_index(g, c);
  const int st1 = g.d[0], st2 = st1 * g.d[1], st3 = st2 * g.d[2];
  Spinor<R> h;
  zero(h);
  hop_in_domain<R, 0, FWD>(g, links, z, L, rhs, s, lc, 1, h);
  hop_in_domain<R, 1, FWD>(g, links, z, L, rhs, s, lc, st1, h);
  hop_in_domain<R, 2, FWD>(g, links, z, L, rhs, s, lc, st2, h);
  hop_in_domain<R, 3, FWD>(g, links, z, L, rhs, s, lc, st3, h);
  if (CM == 1) {
    Spinor<R> t;
    herm_apply<R>(tinv + (size_t)s * HERM_PER_SITE, h, t);
    h = t;
  }
  Spinor<R> v;
  load_spinor(y + spinor_offset(s, L, rhs), v);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    cx<R>& o = (&v.c[0][0])[j];
    const cx<R> a = (&h.c[0][0])[j];
    o = mk(fma(komega, a.re, o.re), fma(komega, a.im, o.im));
  }
  store_spinor(z + spinor_offset(s, L, rhs), v);
}

// ---------------------------------------------------------------------------
// Fused SAP colour sweep with the MR iterations on chip (FP32).
//
// Persistent thread-block clusters walk the (domain of the colour, column
// group) items, NCOL columns per thread.  The DX x DY x DZ x DT domain is cut
// into CX x CY x CZ x CT sub-blocks, one per CTA of the cluster, one thread per
// site; cutting y, z and t gives every CTA the same number of hops that leave
// the domain and of hops into a neighbouring CTA, so no CTA lags at the
// cluster barriers.  A column's hops are summed in one fixed order whatever
// the cut and NCOL, so every launch shape gives the same bits with frozen
// step lengths.  The MR residual of its sites lives in shared memory, double
// buffered so that one cluster barrier per MR step separates the neighbour
// reads of one step from the writes of the next; x and q stay in registers.
// Spinors are stored as 6 float4 planes so consecutive threads read
// consecutive 16-byte words; hops into a neighbouring CTA read its shared
// memory (distributed shared memory).  The first two rows of each site's
// forward links are staged in shared memory once per domain and serve every
// column and MR step.
// The colour's residual r = eta - A psi is formed beforehand by the residual
// kernel (a full-operator stencil over the colour's sites that streams psi
// and eta from HBM with its halo), so the sweep itself only reads r and psi
// and writes psi.  For every column:
//   nmr times: q = A_dom r; omega (per column from the cluster-wide dots, or
//   from the frozen table); x += omega r; r -= omega q,
//   psi += x.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pick4(int mu, int a, int b, int c, int d) {
  return mu == 0 ? a : mu == 1 ? b : mu == 2 ? c : d;
}

// NCOL columns per thread: a thread sweeps NCOL consecutive columns of its
// site at once, so each link is read and completed once for all of them.
template <int DX, int DY, int DZ, int DT, int CX, int CY, int CZ, int CT, int NCOL>
struct SweepShape {
  static constexpr int SX = DX / CX, SY = DY / CY, SZ = DZ / CZ, ST = DT / CT;
  static constexpr int NS = SX * SY * SZ * ST;  // sites per CTA = threads
  static constexpr int CS = CX * CY * CZ * CT;  // CTAs per cluster
  static constexpr int RP = 6 * NCOL;           // float4 planes of one residual buffer
  // two residual buffers, the first two rows of the four forward links of
  // each site (12 float4 planes), partial dots [CS][NCOL][4]
  static constexpr size_t smem_bytes() { return (size_t)NS * (2 * RP + 12) * 16 + CS * NCOL * 4 * sizeof(float); }
};

__device__ __forceinline__ void spinor_to_planes(float4* vS, int NS, int site, const Spinor<float>& v) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const cx<float> a = (&v.c[0][0])[2 * k], b = (&v.c[0][0])[2 * k + 1];
    vS[k * NS + site] = make_float4(a.re, a.im, b.re, b.im);
  }
}
__device__ __forceinline__ void planes_to_spinor(const float4* vS, int NS, int site, Spinor<float>& v) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 t = vS[k * NS + site];
    (&v.c[0][0])[2 * k] = mk(t.x, t.y);
    (&v.c[0][0])[2 * k + 1] = mk(t.z, t.w);
  }
}

// Shared-memory words of any CTA of the cluster by 32-bit shared::cluster
// address: mapa turns a CTA-local shared address into the address of the
// same offset in CTA `rank`; one load instruction then serves hops inside
// the CTA and hops into a neighbouring CTA alike, so warps do not diverge.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ float4 ld_cluster_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

// Asynchronous 16-byte global -> shared copies (cp.async, L1 bypassed),
// waited for by the issuing thread.
__device__ __forceinline__ void cp_async_16(float4* dst, const float4* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The cluster barrier in two halves: arrive publishes this thread's earlier
// shared-memory writes to the cluster (release), wait returns once every
// thread of the cluster has arrived and makes their writes visible (acquire).
// Work between the two halves may read only what this CTA wrote.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Spinor of site `site` from 6 float4 planes of NS sites at cluster address base.
__device__ __forceinline__ void cluster_planes_to_spinor(uint32_t base, int NS, int site, Spinor<float>& v) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 t = ld_cluster_f4(base + (uint32_t)(k * NS + site) * 16u);
    (&v.c[0][0])[2 * k] = mk(t.x, t.y);
    (&v.c[0][0])[2 * k + 1] = mk(t.z, t.w);
  }
}

// The first two rows of an SU(3) link from its 3 float4 planes (link mu of
// site `site`, cluster address base); the third row is rebuilt as the
// complex conjugate of the cross product of the first two (unitarity with
// det = 1).
__device__ __forceinline__ void cluster_planes_to_link12(uint32_t base, int NS, int mu, int site, Link<float>& u) {
  const float4 a = ld_cluster_f4(base + (uint32_t)((mu * 3 + 0) * NS + site) * 16u);
  const float4 b = ld_cluster_f4(base + (uint32_t)((mu * 3 + 1) * NS + site) * 16u);
  const float4 c = ld_cluster_f4(base + (uint32_t)((mu * 3 + 2) * NS + site) * 16u);
  u.m[0][0] = mk(a.x, a.y);
  u.m[0][1] = mk(a.z, a.w);
  u.m[0][2] = mk(b.x, b.y);
  u.m[1][0] = mk(b.z, b.w);
  u.m[1][1] = mk(c.x, c.y);
  u.m[1][2] = mk(c.z, c.w);
  complete_third_row(u);
}

// As cluster_planes_to_link12, from the CTA's own planes.
__device__ __forceinline__ void planes_to_link12(const float4* uS, int NS, int mu, int site, Link<float>& u) {
  const float4 a = uS[(mu * 3 + 0) * NS + site], b = uS[(mu * 3 + 1) * NS + site], c = uS[(mu * 3 + 2) * NS + site];
  u.m[0][0] = mk(a.x, a.y);
  u.m[0][1] = mk(a.z, a.w);
  u.m[0][2] = mk(b.x, b.y);
  u.m[1][0] = mk(b.z, b.w);
  u.m[1][1] = mk(c.x, c.y);
  u.m[1][2] = mk(c.z, c.w);
  complete_third_row(u);
}

// Dirichlet hop sums of the domain operator A_dom over the eight neighbours
// of a site of the domain (hops that leave the domain are dropped) for NCOL
// columns, reading each neighbour's spinors from the (distributed) shared-
// memory planes at cluster address vS (column c at plane 6 c) and the link
// rows from the planes at uS (the site's own forward links; the neighbour's
// for a backward hop), once for all columns.  vS is a CTA-local shared
// address, uS the CTA's link planes already in the cluster window; vL and uL
// are the same planes as pointers, read directly where the hop cannot leave
// the CTA.  sb: coordinates inside the CTA's sub-block, lc: inside the domain.
// The hops are summed in a fixed order (x, y, z, t; forward first), the same
// for every split of the domain and every NCOL.
template <typename SH, int NCOL, int DX, int DY, int DZ, int DT, int CX, int CY, int CZ>
__device__ __forceinline__ void domain_hops(const float4* vL, uint32_t vS, const float4* uL, uint32_t uS, int tid,
                                            int rank, const int sb[4], const int lc[4], Spinor<float> (&acc)[NCOL]) {
  constexpr int NS = SH::NS;
#pragma unroll
  for (int c = 0; c < NCOL; ++c) zero(acc[c]);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int fwd = 1; fwd >= 0; --fwd) {
      const int ext = pick4(mu, DX, DY, DZ, DT);
      const int sub = pick4(mu, SH::SX, SH::SY, SH::SZ, SH::ST);
      const int sub_stride = pick4(mu, 1, SH::SX, SH::SX * SH::SY, SH::SX * SH::SY * SH::SZ);
      const int cta_stride = pick4(mu, 1, CX, CX * CY, CX * CY * CZ);
      const bool leaves = fwd ? (lc[mu] == ext - 1) : (lc[mu] == 0);
      if (leaves) continue;
      // the neighbour is in this CTA or, across a face of the sub-block, at
      // the same position on the far face of the next CTA
      const int sn_sub = sb[mu] + (fwd ? 1 : -1);
      const bool cross = sn_sub < 0 || sn_sub >= sub;
      const int nb = cross ? tid + (fwd ? -(sub - 1) * sub_stride : (sub - 1) * sub_stride)
                           : tid + (fwd ? sub_stride : -sub_stride);
      // A warp covers one (z, t) position of the sub-block (SX * SY >= 32),
      // so in z and t the choice between this CTA and the next is the same
      // for the whole warp: branch, and read this CTA's planes directly.
      // In y it differs inside a warp: one cluster-window load path for all.
      constexpr bool warp_uniform_zt = SH::SX * SH::SY >= 32;
      const bool in_cta = pick4(mu, CX, CY, CZ, SH::CS / (CX * CY * CZ)) == 1 || (mu >= 2 && warp_uniform_zt && !cross);
      const uint32_t other = (uint32_t)(cross ? rank + (fwd ? cta_stride : -cta_stride) : rank);
      Link<float> u;
      if (fwd || in_cta) planes_to_link12(uL, NS, mu, fwd ? tid : nb, u);
      else cluster_planes_to_link12(cluster_addr(uS, other), NS, mu, nb, u);
      const uint32_t vO = in_cta ? 0u : cluster_addr(vS, other);
#pragma unroll
      for (int c = 0; c < NCOL; ++c) {
        Spinor<float> pn;
        if (in_cta) planes_to_spinor(vL + 6 * c * NS, NS, nb, pn);
        else cluster_planes_to_spinor(vO + (uint32_t)(6 * c * NS * 16), NS, nb, pn);
        cx<float> h[2][3], w[2][3];
        const float phase = 1.0f;
        if (fwd) {
          switch (mu) {
            case 0: project<0, -1>(pn, h); link_times<false>(u, h, phase, w); reconstruct_add<0, -1>(acc[c], w); break;
            case 1: project<1, -1>(pn, h); link_times<false>(u, h, phase, w); reconstruct_add<1, -1>(acc[c], w); break;
            case 2: project<2, -1>(pn, h); link_times<false>(u, h, phase, w); reconstruct_add<2, -1>(acc[c], w); break;
            default: project<3, -1>(pn, h); link_times<false>(u, h, phase, w); reconstruct_add<3, -1>(acc[c], w); break;
          }
        } else {
          switch (mu) {
            case 0: project<0, 1>(pn, h); link_times<true>(u, h, phase, w); reconstruct_add<0, 1>(acc[c], w); break;
            case 1: project<1, 1>(pn, h); link_times<true>(u, h, phase, w); reconstruct_add<1, 1>(acc[c], w); break;
            case 2: project<2, 1>(pn, h); link_times<true>(u, h, phase, w); reconstruct_add<2, 1>(acc[c], w); break;
            default: project<3, 1>(pn, h); link_times<true>(u, h, phase, w); reconstruct_add<3, 1>(acc[c], w); break;
          }
        }
      }
    }
  }
}

// CM = 1: the Jacobi-preconditioned clover matrix, every hop sum multiplied by
// T^{-1} of its site (tinv, packed, read through L1)
// H: the residual rin and psi are FP16 spinors with per-(site, column) scales
// rsc, psc (the preconditioner's FP16 storage), else FP32 (rsc, psc unused).
// NCOL: columns per thread; an item is a domain and NCOL consecutive columns
// (when nc is not a multiple of NCOL, the last item's missing columns repeat
// its first one and are not stored).
template <int DX, int DY, int DZ, int DT, int CX, int CY, int CZ, int CT, int CM, bool H, int NCOL>
__global__ void __launch_bounds__(SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>::NS,
                                  (SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>::NS <= 256 && NCOL == 1) ? 2 : 1)
    k_sap_sweep(Geom g, int colour, const cx<float>* __restrict__ links, const void* __restrict__ rin,
                const float* __restrict__ rsc, void* __restrict__ psi, float* __restrict__ psc, int L, int c0, int nc,
                float kappa, int psi_mode, int nmr, int mode, const double* __restrict__ table,
                const float* __restrict__ tinv) {
  using SH = SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>;
  constexpr int NS = SH::NS;
  constexpr int CS = SH::CS;
  constexpr int RP = SH::RP;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float4 sm4[];
  float4* buf0 = sm4;                                       // [NCOL][6][NS] residual
  float4* buf1 = sm4 + RP * NS;                             // [NCOL][6][NS] residual
  float4* uS = sm4 + 2 * RP * NS;                           // [12][NS] link rows 0, 1
  float* red = reinterpret_cast<float*>(sm4 + (2 * RP + 12) * NS);  // [CS][NCOL][4] partial dots
  __shared__ float wsum[NS / 32][NCOL * 3];
  __shared__ float2 oms[MAX_NMR];  // frozen step lengths of the current domain

  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  int sb[4], cb[4], lc[4];
  sb[0] = tid % SH::SX;
  sb[1] = (tid / SH::SX) % SH::SY;
  sb[2] = (tid / (SH::SX * SH::SY)) % SH::SZ;
  sb[3] = tid / (SH::SX * SH::SY * SH::SZ);
  cb[0] = rank % CX;
  cb[1] = (rank / CX) % CY;
  cb[2] = (rank / (CX * CY)) % CZ;
  cb[3] = rank / (CX * CY * CZ);
  lc[0] = cb[0] * SH::SX + sb[0];
  lc[1] = cb[1] * SH::SY + sb[1];
  lc[2] = cb[2] * SH::SZ + sb[2];
  lc[3] = cb[3] * SH::ST + sb[3];
  const int ndc = g.nd / 2;
  // persistent clusters: the (domain, column group) items of this colour,
  // domain major, are cut into one contiguous range per cluster
  const int nclu = gridDim.x / CS;
  const int cid = blockIdx.x / CS;
  const int ngrp = (nc + NCOL - 1) / NCOL;  // column groups of the columns c0 .. c0 + nc - 1
  const long long nitems = (long long)ndc * ngrp;
  const int item0 = (int)(nitems * cid / nclu);
  const int item1 = (int)(nitems * (cid + 1) / nclu);
  const uint32_t uA = cluster_addr(smem_addr(uS), (uint32_t)rank);  // own link planes, cluster window
  // the column of slot j of group grp (a missing one repeats the first)
  auto column = [&](int grp, int j) { return c0 + grp * NCOL + ((grp * NCOL + j < nc) ? j : 0); };

  // A buffer is written only after the cluster barrier that follows the last
  // reads of it by other CTAs; every write is followed by a barrier before
  // the buffer is read.  Each thread arrives at the barrier once its writes
  // are done and waits just before the hops that read the other CTAs.
  float4* cur = buf0;
  float4* nxt = buf1;
  int k = -1, s = 0;
  int c[4];
  // With frozen step lengths the last MR step applies no operator and leaves
  // the buffer nxt idle (no CTA reads it after the barrier that ended the
  // step before): there the next item's FP32 residual is copied into nxt with
  // asynchronous 16-byte copies, so its HBM latency overlaps the step and the
  // psi update instead of stalling the cluster at the next item's start.
  bool have_rn = false;
  for (int item = item0; item < item1; ++item) {
    const int kk = item / ngrp;
    const int grp = item - kk * ngrp;
    if (kk != k) {
      k = kk;  // a new domain of this colour
      int b[4];
      colour_domain(g, colour, k, b);
      c[0] = b[0] * DX + lc[0];
      c[1] = b[1] * DY + lc[1];
      c[2] = b[2] * DZ + lc[2];
      c[3] = b[3] * DT + lc[3];
      s = site_index(g, c);
      if (item != item0) cluster.sync();  // no CTA still reads the previous domain's links
      // the first two rows of this site's four forward links, for all columns
      // of the domain; the barrier after the first staging of r makes them
      // visible to the cluster
      const float2* gl = reinterpret_cast<const float2*>(links + (size_t)s * 36);
#pragma unroll
      for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float2 v0 = __ldg(gl + mu * 9 + 2 * q), v1 = __ldg(gl + mu * 9 + 2 * q + 1);
          uS[(mu * 3 + q) * NS + tid] = make_float4(v0.x, v0.y, v1.x, v1.y);
        }
      // the domain's frozen step lengths, rounded to FP32 once per domain
      if (mode != 0)
        for (int it = tid; it < nmr; it += NS) {
          const double* tb = table + ((size_t)it * ndc + k) * 2;
          oms[it] = make_float2((float)tb[0], (float)tb[1]);
        }
    }
    // the colour's residual at entry: eta itself when psi = 0, else
    // eta - A psi formed beforehand by the residual kernel
    if (have_rn) {
      cp_async_wait_all();  // this thread's copies of r0 into nxt have landed
    } else {
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const size_t off = spinor_offset(s, L, column(grp, j));
        Spinor<float> r0;
        if (H) load_spinor_h(static_cast<const __half2*>(rin) + off, __ldg(rsc + off / 12), r0);
        else load_spinor(static_cast<const cx<float>*>(rin) + off, r0);
        spinor_to_planes(nxt + 6 * j * NS, NS, tid, r0);
      }
    }
    have_rn = false;
    cluster_arrive();  // r0 (and, for a new domain, this CTA's links and step lengths) written
    { float4* t = cur; cur = nxt; nxt = t; }
    Spinor<float> x[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) zero(x[j]);

    // the MR steps that apply the operator: all of them with per-column step
    // lengths, all but the last with frozen ones
    const int nop = (mode == 0) ? nmr : nmr - 1;
    for (int it = 0; it < nop; ++it) {
      const bool last = (it == nmr - 1);
      Spinor<float> q[NCOL];
      cluster_wait();  // the residual planes of every CTA
      domain_hops<SH, NCOL, DX, DY, DZ, DT, CX, CY, CZ>(cur, smem_addr(cur), uS, uA, tid, rank, sb, lc, q);
      if (CM == 1) {
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          Spinor<float> h;
          herm_apply<float>(tinv + (size_t)s * HERM_PER_SITE, q[j], h);
          q[j] = h;
        }
      }
      cx<float> om[NCOL];
      if (mode == 0) {
        float dots[NCOL][3];
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          Spinor<float> rv;
          planes_to_spinor(cur + 6 * j * NS, NS, tid, rv);
          float nre = 0, nim = 0, den = 0;
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            cx<float>& o = (&q[j].c[0][0])[e];
            const cx<float> v = (&rv.c[0][0])[e];
            o = mk(fmaf(-kappa, o.re, v.re), fmaf(-kappa, o.im, v.im));
            nre = fmaf(o.re, v.re, fmaf(o.im, v.im, nre));
            nim = fmaf(o.re, v.im, fmaf(-o.im, v.re, nim));
            den = fmaf(o.re, o.re, fmaf(o.im, o.im, den));
          }
          dots[j][0] = nre;
          dots[j][1] = nim;
          dots[j][2] = den;
        }
        // CTA reduction: warp shuffles, then the warps' sums in a fixed order
#pragma unroll
        for (int j = 0; j < NCOL; ++j)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dots[j][d] += __shfl_xor_sync(0xffffffffu, dots[j][d], o);
            if ((tid & 31) == 0) wsum[tid >> 5][j * 3 + d] = dots[j][d];
          }
        __syncthreads();
        if (tid < NCOL * 3) {
          float a = 0;
          for (int w = 0; w < NS / 32; ++w) a += wsum[w][tid];
          red[rank * NCOL * 4 + (tid / 3) * 4 + tid % 3] = a;
        }
        cluster.sync();
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          double tre = 0, tim = 0, tden = 0;
          for (int q2 = 0; q2 < CS; ++q2) {
            const float* rr = cluster.map_shared_rank(red, q2) + q2 * NCOL * 4 + j * 4;
            tre += rr[0];
            tim += rr[1];
            tden += rr[2];
          }
          om[j] = tden > 0 ? mk((float)(tre / tden), (float)(tim / tden)) : mk(0.0f, 0.0f);
        }
      } else {
        const float2 o2 = oms[it];
#pragma unroll
        for (int j = 0; j < NCOL; ++j) om[j] = mk(o2.x, o2.y);
      }
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        Spinor<float> rv;
        planes_to_spinor(cur + 6 * j * NS, NS, tid, rv);
        if (mode != 0) {
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            cx<float>& o = (&q[j].c[0][0])[e];
            const cx<float> v = (&rv.c[0][0])[e];
            o = mk(fmaf(-kappa, o.re, v.re), fmaf(-kappa, o.im, v.im));
          }
        }
#pragma unroll
        for (int e = 0; e < 12; ++e) cmac((&x[j].c[0][0])[e], om[j], (&rv.c[0][0])[e]);
        if (!last) {
          const cx<float> mom = mk(-om[j].re, -om[j].im);
#pragma unroll
          for (int e = 0; e < 12; ++e) cmac((&rv.c[0][0])[e], mom, (&q[j].c[0][0])[e]);
          spinor_to_planes(nxt + 6 * j * NS, NS, tid, rv);
        }
      }
      if (!last) {
        cluster_arrive();
        float4* t = cur; cur = nxt; nxt = t;
      }
    }
    // psi += x for the group's columns.  With frozen step lengths the last MR
    // step applies no operator: psi's loads are issued before its wait for
    // the other CTAs, which hides their latency, and the step only adds
    // omega r to x.
    Spinor<float> pv[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      const size_t off = spinor_offset(s, L, c0 + grp * NCOL + j);
      if (psi_mode == 1 || grp * NCOL + j >= nc) zero(pv[j]);
      else if (H) load_spinor_h(static_cast<const __half2*>(psi) + off, psc[off / 12], pv[j]);
      else load_spinor(static_cast<const cx<float>*>(psi) + off, pv[j]);
    }
    if (mode != 0) {
      cluster_wait();  // no CTA reads nxt any more
      if (!H && item + 1 < item1) {
        // the next item: the next column group of this site, or the first
        // one of the next domain
        const int kn = (item + 1) / ngrp;
        const int gn = item + 1 - kn * ngrp;
        int sn = s;
        if (kn != kk) {
          int b[4], cn[4];
          colour_domain(g, colour, kn, b);
          cn[0] = b[0] * DX + lc[0];
          cn[1] = b[1] * DY + lc[1];
          cn[2] = b[2] * DZ + lc[2];
          cn[3] = b[3] * DT + lc[3];
          sn = site_index(g, cn);
        }
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          const size_t offn = spinor_offset(sn, L, column(gn, j));
          const float4* src = reinterpret_cast<const float4*>(static_cast<const cx<float>*>(rin) + offn);
#pragma unroll
          for (int e = 0; e < 6; ++e) cp_async_16(nxt + (6 * j + e) * NS + tid, src + e);
        }
        cp_async_commit();
        have_rn = true;
      }
      const float2 o2 = oms[nmr - 1];
      const cx<float> om = mk(o2.x, o2.y);
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        Spinor<float> rv;
        planes_to_spinor(cur + 6 * j * NS, NS, tid, rv);
#pragma unroll
        for (int e = 0; e < 12; ++e) cmac((&x[j].c[0][0])[e], om, (&rv.c[0][0])[e]);
      }
    }
#pragma unroll
    for (int j = 0; j < NCOL; ++j) {
      if (grp * NCOL + j >= nc) break;
      const size_t off = spinor_offset(s, L, c0 + grp * NCOL + j);
#pragma unroll
      for (int e = 0; e < 12; ++e) (&pv[j].c[0][0])[e] = (&pv[j].c[0][0])[e] + (&x[j].c[0][0])[e];
      if (H) store_spinor_h(static_cast<__half2*>(psi) + off, psc + off / 12, pv[j]);
      else store_spinor(static_cast<cx<float>*>(psi) + off, pv[j]);
    }
    // the next item writes its residual into nxt: the last reads of nxt by
    // other CTAs were fenced by the barrier that followed them
  }
  // no CTA of the cluster may exit while others still read its shared memory
  cluster.sync();
}

// sets the sweep kernel's shared-memory and cluster attributes and returns
// how many of its clusters the GPU holds at once
template <int DX, int DY, int DZ, int DT, int CX, int CY, int CZ, int CT, int CM, bool H, int NCOL>
int sweep_setup(cudaLaunchConfig_t cfg) {
  using SH = SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>;
  auto kern = k_sap_sweep<DX, DY, DZ, DT, CX, CY, CZ, CT, CM, H, NCOL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::smem_bytes());
  if (SH::CS > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cfg.gridDim = dim3((unsigned)SH::CS);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

template <int DX, int DY, int DZ, int DT, int CX, int CY, int CZ, int CT, int CM, bool H, int NCOL>
bool launch_sweep(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const void* rin, const float* rsc,
                  void* psi, float* psc, int L, int c0, int nc, double kappa, int psi_mode, int nmr, int mode,
                  const double* table, const float* tinv) {
  using SH = SweepShape<DX, DY, DZ, DT, CX, CY, CZ, CT, NCOL>;
  auto kern = k_sap_sweep<DX, DY, DZ, DT, CX, CY, CZ, CT, CM, H, NCOL>;
  const size_t shm = SH::smem_bytes();
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(SH::NS);
  cfg.dynamicSmemBytes = shm;
  cfg.stream = ex.stream;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = SH::CS;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  // one persistent cluster per cluster slot of the GPU (clusters must fit
  // in one GPC, so fewer than SMs / CS may be resident at once); set up once
  // per process, thread-safely (contexts may run on several host threads)
  static const int max_clusters = sweep_setup<DX, DY, DZ, DT, CX, CY, CZ, CT, CM, H, NCOL>(cfg);
  const long long nitems = (long long)(g.nd / 2) * ((nc + NCOL - 1) / NCOL);
  const int nclu = (int)std::min<long long>(max_clusters, nitems);
  cfg.gridDim = dim3((unsigned)(SH::CS * nclu));
  cudaLaunchKernelEx(&cfg, kern, g, colour, links, rin, rsc, psi, psc, L, c0, nc, (float)kappa, psi_mode, nmr, mode,
                     table, tinv);
  ++*ex.launches;
  return true;
}

template <int CM, bool H>
bool launch_sweep8(int shape, const Exec& ex, const Geom& g, int colour, const cx<float>* links, const void* rin,
                   const float* rsc, void* psi, float* psc, int L, int c0, int nc, double kappa, int psi_mode, int nmr,
                   int mode, const double* table, const float* tinv) {
  if (shape == 1)
    return launch_sweep<8, 8, 8, 8, 1, 2, 2, 4, CM, H, 2>(ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa,
                                                          psi_mode, nmr, mode, table, tinv);
  if (shape == 2)
    return launch_sweep<8, 8, 8, 8, 1, 2, 2, 4, CM, H, 1>(ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa,
                                                          psi_mode, nmr, mode, table, tinv);
  return launch_sweep<8, 8, 8, 8, 1, 2, 2, 2, CM, H, 1>(ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa,
                                                        psi_mode, nmr, mode, table, tinv);
}

// shape: one of the 8^4 launch shapes (tune.h); 4^4 domains have one (a
// single CTA per domain)
template <bool H>
bool sweep_dispatch(int shape, const Exec& ex, const Geom& g, int colour, const cx<float>* links, const void* rin,
                    const float* rsc, void* psi, float* psc, int L, int c0, int nc, double kappa, int psi_mode, int nmr,
                    int mode, const double* table, const float* tinv) {
  if (g.blk[0] == 8) {
    if (tinv)
      return launch_sweep8<1, H>(shape, ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa, psi_mode, nmr,
                                 mode, table, tinv);
    return launch_sweep8<0, H>(shape, ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa, psi_mode, nmr, mode,
                               table, nullptr);
  }
  if (tinv)
    return launch_sweep<4, 4, 4, 4, 1, 1, 1, 1, 1, H, 1>(ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa,
                                                         psi_mode, nmr, mode, table, tinv);
  return launch_sweep<4, 4, 4, 4, 1, 1, 1, 1, 0, H, 1>(ex, g, colour, links, rin, rsc, psi, psc, L, c0, nc, kappa,
                                                       psi_mode, nmr, mode, table, nullptr);
}

// the launch shape of the sweep for this lattice, storage and L: the one
// MBICG_SWEEP_SHAPE names, else the tuned one, else 0
int sweep_shape(const Geom& g, bool half, bool clover, int L) {
  if (g.blk[0] != 8) return 0;
  if (const char* e = getenv("MBICG_SWEEP_SHAPE")) {
    const int v = atoi(e);
    if (e[0] >= '0' && e[0] <= '9' && v < SWEEP_SHAPES) return v;
  }
  int idx;
  if (tune_table().lookup(sweep_key(half, clover, g.d, L), &idx) && idx >= 0 && idx < SWEEP_SHAPES) return idx;
  return 0;
}

}  // namespace

bool sap_sweep_fusable(const Geom& g, int mode) {
  if (!(mode == 0 || mode == 3) || !g.su3) return false;  // the kernel rebuilds the third link row
  const int* bk = g.blk;
  return (bk[0] == 8 && bk[1] == 8 && bk[2] == 8 && bk[3] == 8) || (bk[0] == 4 && bk[1] == 4 && bk[2] == 4 && bk[3] == 4);
}

bool sap_sweep_fused(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const cx<float>* eta,
                     cx<float>* psi, int L, double kappa, int psi_mode, int nmr, int mode, const double* table,
                     const float* tinv, int c0, int nc) {
  if (!sap_sweep_fusable(g, mode)) return false;
  return sweep_dispatch<false>(sweep_shape(g, false, tinv != nullptr, L), ex, g, colour, links, eta, nullptr, psi,
                               nullptr, L, c0, nc > 0 ? nc : L, kappa, psi_mode, nmr, mode, table, tinv);
}

bool sap_sweep_fused_h(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const __half2* rin,
                       const float* rsc, __half2* psi, float* psc, int L, double kappa, int psi_mode, int nmr,
                       int mode, const double* table, const float* tinv, int c0, int nc) {
  if (!sap_sweep_fusable(g, mode)) return false;
  return sweep_dispatch<true>(sweep_shape(g, true, tinv != nullptr, L), ex, g, colour, links, rin, rsc, psi, psc, L, c0,
                              nc > 0 ? nc : L, kappa, psi_mode, nmr, mode, table, tinv);
}

void tune_sap_sweep(const Exec& ex, const Geom& g, const cx<float>* links, void* rin, float* rsc, void* psi, float* psc,
                    int L, double kappa, int nmr, const double* table, bool half, const float* tinv) {
  if (g.blk[0] != 8 || !sap_sweep_fusable(g, 3)) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ex.stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  const char* tr = getenv("MBICG_TRACE");
  const std::string key = sweep_key(half, tinv != nullptr, g.d, L);
  int known;
  if (tune_table().lookup(key, &known)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return;
  }
  // defined contents for the timing runs (zeros; the runs overwrite psi)
  const size_t n = (size_t)g.V * 12 * L;
  if (cudaMemsetAsync(rin, 0, n * (half ? sizeof(__half2) : sizeof(cx<float>)), ex.stream) != cudaSuccess ||
      cudaMemsetAsync(psi, 0, n * (half ? sizeof(__half2) : sizeof(cx<float>)), ex.stream) != cudaSuccess ||
      (half && (cudaMemsetAsync(rsc, 0, sizeof(float) * g.V * L, ex.stream) != cudaSuccess ||
                cudaMemsetAsync(psc, 0, sizeof(float) * g.V * L, ex.stream) != cudaSuccess))) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return;
  }
  tune_table().pick(key, SWEEP_SHAPES, [&](int i) -> double {
    cudaEventRecord(e0, ex.stream);
    if (half)
      sweep_dispatch<true>(i, ex, g, 0, links, rin, rsc, psi, psc, L, 0, L, kappa, 2, nmr, 3, table, tinv);
    else
      sweep_dispatch<false>(i, ex, g, 0, links, rin, nullptr, psi, nullptr, L, 0, L, kappa, 2, nmr, 3, table, tinv);
    cudaEventRecord(e1, ex.stream);
    float ms = -1.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return -1.0;
    if (tr && tr[0] == '1') fprintf(stderr, "mbicg: tune %s shape %d: %.3f ms\n", key.c_str(), i, ms);
    return ms;
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (const char* p = getenv("MBICG_TUNE_FILE")) tune_table().save(p);
}

void sap_residual_h(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const __half2* eta,
                    const float* esc, const __half2* psi, const float* psc, __half2* r, float* rsc, int L, double kappa,
                    const float* tinv, int c0, int nc) {
  if (nc <= 0) nc = L;
  const int S = sap_sites_per_cta(g, nc, false);
  const int nslot = (g.nd / 2) * g.Vd;
  if (tinv)
    k_sap_residual_h<1><<<(unsigned)(nslot / S), dim3(nc, S), 0, ex.stream>>>(g, colour, links, eta, esc, psi, psc,
                                                                             r, rsc, L, c0, (float)kappa, tinv);
  else
    k_sap_residual_h<0><<<(unsigned)(nslot / S), dim3(nc, S), 0, ex.stream>>>(g, colour, links, eta, esc, psi, psc,
                                                                             r, rsc, L, c0, (float)kappa, nullptr);
  ++*ex.launches;
}

namespace {

int pow2_floor(int v) {
  int p = 1;
  while (p * 2 <= v) p *= 2;
  return p;
}

}  // namespace

int sap_sites_per_cta(const Geom& g, int L, bool fp64) {
  int S = pow2_floor((fp64 ? 256 : 384) / L);
  while (S > 1 && (g.Vd % S) != 0) S >>= 1;
  return S;
}

// one launch of the operator in configuration cfg (tune.h)
// links12: the FP32 links as their first two rows (SU(3) fields), used by the
// Wilson operator in FP32 when given
template <typename R>
void launch_dslash(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* in, cx<R>* out, int L,
                   double kappa, DslashConfig cfg, const R* clov, int cm, const cx<float>* links12) {
  const int S = cfg.S;
  const dim3 block(L, S);
  const int grid = (g.V + S - 1) / S;
  const int slice = g.d[0] * g.d[1] * g.d[2];
  const bool slabs = cfg.order == 1 && slice % S == 0 && g.d[3] % 8 == 0;
  const int ws = slabs ? slice / S : 0, tt = slabs ? 8 : 1;
  if constexpr (std::is_same<R, float>::value) {
    if (cm == 0 && links12) {
      k_dslash_full<float, 0, true><<<(unsigned)grid, block, 0, ex.stream>>>(g, links12, in, out, L, (float)kappa,
                                                                             nullptr, ws, tt);
      ++*ex.launches;
      return;
    }
  }
  if (cm == 1)
    k_dslash_full<R, 1><<<(unsigned)grid, block, 0, ex.stream>>>(g, links, in, out, L, (R)kappa, clov, ws, tt);
  else if (cm == 2)
    k_dslash_full<R, 2><<<(unsigned)grid, block, 0, ex.stream>>>(g, links, in, out, L, (R)kappa, clov, ws, tt);
  else
    k_dslash_full<R, 0><<<(unsigned)grid, block, 0, ex.stream>>>(g, links, in, out, L, (R)kappa, nullptr, ws, tt);
  ++*ex.launches;
}

// the configuration the tuner chose for this operator, else the default: the
// most sites per CTA, in time slabs where they tile the time slices
template <typename R>
DslashConfig dslash_config(const Geom& g, int L) {
  const std::vector<DslashConfig> cand = dslash_candidates(g.d, L, max_cta<R>());
  int idx;
  if (tune_table().lookup(dslash_key((int)sizeof(R), g.d, L), &idx) && idx >= 0 && idx < (int)cand.size())
    return cand[idx];
  return cand.size() > 1 && cand[1].S == cand[0].S ? cand[1] : cand[0];
}

template <typename R>
void dslash_full(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* in, cx<R>* out, int L,
                 double kappa, const R* clov, int cm, const cx<float>* links12) {
  launch_dslash<R>(ex, g, links, in, out, L, kappa, dslash_config<R>(g, L), clov, cm, links12);
}

template <typename R>
void tune_dslash(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* in, cx<R>* out, int L,
                 double kappa, const cx<float>* links12) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ex.stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  const std::vector<DslashConfig> cand = dslash_candidates(g.d, L, max_cta<R>());
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  tune_table().pick(dslash_key((int)sizeof(R), g.d, L), (int)cand.size(), [&](int i) -> double {
    cudaEventRecord(e0, ex.stream);
    launch_dslash<R>(ex, g, links, in, out, L, kappa, cand[i], nullptr, 0, links12);
    cudaEventRecord(e1, ex.stream);
    float ms = -1.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return -1.0;
    return ms;
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (const char* p = getenv("MBICG_TUNE_FILE")) tune_table().save(p);
}

template <typename R>
void sap_residual(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const cx<R>* eta,
                  const cx<R>* psi, cx<R>* r, int L, double kappa, bool psi_zero, const R* tinv, int c0, int nc,
                  const cx<float>* links12) {
  if (nc <= 0) nc = L;
  const int S = sap_sites_per_cta(g, nc, sizeof(R) == 8);
  const int nslot = (g.nd / 2) * g.Vd;
  if constexpr (std::is_same<R, float>::value) {
    if (!tinv && links12) {
      k_sap_residual<float, 0, true><<<(unsigned)(nslot / S), dim3(nc, S), 0, ex.stream>>>(
          g, colour, links12, eta, psi, r, L, c0, (float)kappa, psi_zero ? 1 : 0, nullptr);
      ++*ex.launches;
      return;
    }
  }
  if (tinv)
    k_sap_residual<R, 1><<<(unsigned)(nslot / S), dim3(nc, S), 0, ex.stream>>>(g, colour, links, eta, psi, r, L, c0,
                                                                                (R)kappa, psi_zero ? 1 : 0, tinv);
  else
    k_sap_residual<R, 0><<<(unsigned)(nslot / S), dim3(nc, S), 0, ex.stream>>>(g, colour, links, eta, psi, r, L, c0,
                                                                                (R)kappa, psi_zero ? 1 : 0, nullptr);
  ++*ex.launches;
}

template <typename R>
void sap_domain_apply(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const cx<R>* r,
                      cx<R>* q, double* dots, int L, double kappa, int* nchunk_out, const R* tinv) {
  const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
  const int nchunk = g.Vd / S;
  const int nslot = (g.nd / 2) * g.Vd;
  const size_t shm = dots ? sizeof(R) * 3 * S * L : 0;
  if (tinv)
    k_sap_domain_apply<R, 1><<<(unsigned)(nslot / S), dim3(L, S), shm, ex.stream>>>(g, colour, links, r, q, dots,
                                                                                    L, (R)kappa, nchunk, tinv);
  else
    k_sap_domain_apply<R, 0><<<(unsigned)(nslot / S), dim3(L, S), shm, ex.stream>>>(g, colour, links, r, q, dots,
                                                                                    L, (R)kappa, nchunk, nullptr);
  ++*ex.launches;
  if (nchunk_out) *nchunk_out = nchunk;
}

template <typename R>
void ssor_level(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const R* tinv, const cx<R>* y,
                cx<R>* z, int L, double komega, const int* local, int count, bool fwd) {
  const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
  const int n = (g.nd / 2) * count;
  const unsigned grid = (unsigned)((n + S - 1) / S);
  const dim3 block(L, S);
  if (tinv) {
    if (fwd) k_ssor_level<R, 1, true><<<grid, block, 0, ex.stream>>>(g, colour, links, tinv, y, z, L, (R)komega, local, count);
    else k_ssor_level<R, 1, false><<<grid, block, 0, ex.stream>>>(g, colour, links, tinv, y, z, L, (R)komega, local, count);
  } else {
    if (fwd) k_ssor_level<R, 0, true><<<grid, block, 0, ex.stream>>>(g, colour, links, nullptr, y, z, L, (R)komega, local, count);
    else k_ssor_level<R, 0, false><<<grid, block, 0, ex.stream>>>(g, colour, links, nullptr, y, z, L, (R)komega, local, count);
  }
  ++*ex.launches;
}

#define INST(R)                                                                                          \
  template void dslash_full<R>(const Exec&, const Geom&, const cx<R>*, const cx<R>*, cx<R>*, int, double,  \
                               const R*, int, const cx<float>*);                                        \
  template void tune_dslash<R>(const Exec&, const Geom&, const cx<R>*, const cx<R>*, cx<R>*, int, double,  \
                               const cx<float>*);                                                       \
  template void sap_residual<R>(const Exec&, const Geom&, int, const cx<R>*, const cx<R>*, const cx<R>*,   \
                                cx<R>*, int, double, bool, const R*, int, int, const cx<float>*);         \
  template void sap_domain_apply<R>(const Exec&, const Geom&, int, const cx<R>*, const cx<R>*, cx<R>*,     \
                                    double*, int, double, int*, const R*);                                \
  template void ssor_level<R>(const Exec&, const Geom&, int, const cx<R>*, const R*, const cx<R>*, cx<R>*, \
                              int, double, const int*, int, bool);
INST(float)
INST(double)
#undef INST

}  // namespace mbicg
