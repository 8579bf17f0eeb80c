// clover.cu — the clover term of the O(a)-improved Wilson-Dirac matrix and its
// Jacobi preconditioning (Sec. 2.2, the division by 1 + clover term):
//   D_c = T - kappa H,   T_x = 1 + kappa C_x,
//   C_x = i c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
//   F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^dagger) / 8,
// with Q_{mu nu}(x) the four plaquettes of the (mu, nu) plane that start and
// end at x, all traversed mu before nu (no trace subtracted; links carry no
// boundary phase).  A = T^{-1} D_c = 1 - kappa T^{-1} H is the matrix the
// solver and the SAP preconditioner work with.
//
// In the chiral basis sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] is
// diag(s+, s-) with 2 x 2 blocks that are signed Pauli matrices, so C and
// T^{-1} are two Hermitian 6 x 6 blocks per site (packed, herm_off).  C is
// computed once per gauge field and c_sw in FP64; T^{-1} once per kappa, by
// Gauss-Jordan elimination with partial pivoting of each 6 x 6 block in FP64,
// then rounded to FP32 for the FP32 operator.
#include "internal.h"

namespace mbicg {

namespace {

// sigma_{mu nu} for the planes (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): which
// Pauli matrix and its sign in the block of spins 0-1 and of spins 2-3
struct SigmaBlock {
  int pauli;
  int sign[2];
};
__constant__ SigmaBlock kSigma[6] = {{3, {-1, -1}}, {2, {1, 1}}, {1, {1, -1}},
                                     {1, {-1, -1}}, {2, {1, -1}}, {3, {1, -1}}};

__device__ __forceinline__ cx<double> pauli(int k, int s, int t) {
  if (k == 1) return mk(s != t ? 1.0 : 0.0, 0.0);
  if (k == 2) return s == t ? mk(0.0, 0.0) : mk(0.0, s == 0 ? -1.0 : 1.0);
  return s != t ? mk(0.0, 0.0) : mk(s == 0 ? 1.0 : -1.0, 0.0);
}

// o = a b for 3 x 3 colour matrices, each factor daggered on request
__device__ void mul3(const cx<double>* a, bool da, const cx<double>* b, bool db, cx<double>* o) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cx<double> acc = mk(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const cx<double> x = da ? conjg(a[k * 3 + i]) : a[i * 3 + k];
        const cx<double> y = db ? conjg(b[j * 3 + k]) : b[k * 3 + j];
        cmac(acc, x, y);
      }
      o[i * 3 + j] = acc;
    }
}

// q += l0 l1 l2 l3 (each link daggered where d says so)
__device__ void add_loop(const cx<double>* l0, bool d0, const cx<double>* l1, bool d1, const cx<double>* l2,
                         bool d2, const cx<double>* l3, bool d3, cx<double>* q) {
  cx<double> t1[9], t2[9], t3[9];
  mul3(l0, d0, l1, d1, t1);
  mul3(t1, false, l2, d2, t2);
  mul3(t2, false, l3, d3, t3);
  for (int k = 0; k < 9; ++k) q[k] = q[k] + t3[k];
}

__device__ __forceinline__ int shifted(const Geom& g, const int c[4], int mu, int dm, int nu, int dn) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  n[mu] = (n[mu] + dm + g.d[mu]) % g.d[mu];
  n[nu] = (n[nu] + dn + g.d[nu]) % g.d[nu];
  return site_index(g, n);
}

// C of every site, packed (72 doubles per site); one thread per site
__global__ void k_clover_field(Geom g, const cx<double>* __restrict__ U, double csw, double* __restrict__ C) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    double out[HERM_PER_SITE];
    for (int k = 0; k < HERM_PER_SITE; ++k) out[k] = 0.0;
    auto link = [&](int site, int dir) { return U + ((size_t)site * 4 + dir) * 9; };
    int plane = 0;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
        const int xp = shifted(g, c, mu, 1, nu, 0), xn = shifted(g, c, mu, 0, nu, 1);
        const int xm = shifted(g, c, mu, -1, nu, 0), xd = shifted(g, c, mu, 0, nu, -1);
        const int xmd = shifted(g, c, mu, -1, nu, -1), xmn = shifted(g, c, mu, -1, nu, 1);
        const int xpd = shifted(g, c, mu, 1, nu, -1);
        cx<double> Q[9];
        for (int k = 0; k < 9; ++k) Q[k] = mk(0.0, 0.0);
        // right, up, left, down
        add_loop(link(s, mu), false, link(xp, nu), false, link(xn, mu), true, link(s, nu), true, Q);
        // up, left, down, right
        add_loop(link(s, nu), false, link(xmn, mu), true, link(xm, nu), true, link(xm, mu), false, Q);
        // left, down, right, up
        add_loop(link(xm, mu), true, link(xmd, nu), true, link(xmd, mu), false, link(xd, nu), false, Q);
        // down, right, up, left
        add_loop(link(xd, nu), true, link(xd, mu), false, link(xpd, nu), false, link(s, mu), true, Q);
        const SigmaBlock sb = kSigma[plane];
        for (int b = 0; b < 2; ++b)
          for (int sp = 0; sp < 2; ++sp)
            for (int tp = 0; tp < 2; ++tp) {
              const cx<double> pm = pauli(sb.pauli, sp, tp);
              if (pm.re == 0.0 && pm.im == 0.0) continue;
              const cx<double> sg = (double)sb.sign[b] * pm;
              for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb) {
                  const int i = 3 * sp + a, j = 3 * tp + bb;
                  if (i > j) continue;  // the Hermitian partner of (j, i)
                  const cx<double> F = 0.125 * (Q[a * 3 + bb] - conjg(Q[bb * 3 + a]));
                  const cx<double> v = times_i(csw * (sg * F));
                  if (i == j) {
                    out[36 * b + i] += v.re;
                  } else {
                    const int o = 36 * b + herm_off(i, j);
                    out[o] += v.re;
                    out[o + 1] += v.im;
                  }
                }
            }
      }
    double* dst = C + (size_t)s * HERM_PER_SITE;
    for (int k = 0; k < HERM_PER_SITE; ++k) dst[k] = out[k];
  }
}

// Per 6 x 6 block (one thread each): T = 1 + kappa C, T^{-1} by Gauss-Jordan
// elimination with partial pivoting, packed into Ti64 and (rounded) Ti32;
// C32 = C rounded to FP32.  A singular block sets bit 0 of *status.
__global__ void k_clover_terms(long long nblk, const double* __restrict__ C, double kappa,
                               double* __restrict__ Ti64, float* __restrict__ Ti32, float* __restrict__ C32,
                               int* __restrict__ status) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nblk;
       q += (long long)gridDim.x * blockDim.x) {
    const double* cb = C + q * 36;
    cx<double> a[6][6], inv[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        inv[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
        if (i == j) {
          a[i][j] = mk(1.0 + kappa * cb[i], 0.0);
        } else {
          const int o = herm_off(i < j ? i : j, i < j ? j : i);
          a[i][j] = mk(kappa * cb[o], (i < j ? kappa : -kappa) * cb[o + 1]);
        }
      }
    bool ok = true;
    for (int k = 0; k < 6 && ok; ++k) {
      int p = k;
      double best = a[k][k].re * a[k][k].re + a[k][k].im * a[k][k].im;
      for (int r = k + 1; r < 6; ++r) {
        const double m = a[r][k].re * a[r][k].re + a[r][k].im * a[r][k].im;
        if (m > best) { best = m; p = r; }
      }
      if (!(best > 0.0)) { ok = false; break; }
      if (p != k)
        for (int j = 0; j < 6; ++j) {
          const cx<double> t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t;
          const cx<double> u = inv[k][j]; inv[k][j] = inv[p][j]; inv[p][j] = u;
        }
      const cx<double> rp = mk(a[k][k].re / best, -a[k][k].im / best);  // 1 / pivot
      for (int j = 0; j < 6; ++j) {
        a[k][j] = a[k][j] * rp;
        inv[k][j] = inv[k][j] * rp;
      }
      for (int r = 0; r < 6; ++r) {
        if (r == k) continue;
        const cx<double> f = a[r][k];
        for (int j = 0; j < 6; ++j) {
          a[r][j] = a[r][j] - f * a[k][j];
          inv[r][j] = inv[r][j] - f * inv[k][j];
        }
      }
    }
    if (!ok) atomicOr(status, 1);
    double* t64 = Ti64 + q * 36;
    float* t32 = Ti32 + q * 36;
    for (int i = 0; i < 6; ++i) {
      t64[i] = ok ? inv[i][i].re : 0.0;
      for (int j = i + 1; j < 6; ++j) {
        const int o = herm_off(i, j);
        t64[o] = ok ? inv[i][j].re : 0.0;
        t64[o + 1] = ok ? inv[i][j].im : 0.0;
      }
    }
    for (int k = 0; k < 36; ++k) {
      t32[k] = (float)t64[k];
      C32[q * 36 + k] = (float)cb[k];
    }
  }
}

// out = M in on an ABI-layout block [site][spin][colour][rhs] (FP64), one
// thread per (site, rhs); in and out may alias
__global__ void k_clover_abi(long long nsite, int L, const double* __restrict__ M, const cx<double>* in,
                             cx<double>* out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsite * L) return;
  const long long site = idx / L;
  const int rhs = (int)(idx - site * L);
  Spinor<double> x, y;
  for (int k = 0; k < 12; ++k) (&x.c[0][0])[k] = in[(site * 12 + k) * L + rhs];
  herm_apply<double>(M + site * HERM_PER_SITE, x, y);
  for (int k = 0; k < 12; ++k) out[(site * 12 + k) * L + rhs] = (&y.c[0][0])[k];
}

}  // namespace

void clover_field(const Exec& ex, const Geom& g, const cx<double>* U64, double csw, double* C64) {
  const int grid = (int)std::min<long long>((g.V + 127) / 128, 8 * 152);
  k_clover_field<<<grid, 128, 0, ex.stream>>>(g, U64, csw, C64);
  ++*ex.launches;
}

void clover_terms(const Exec& ex, long long nsite, const double* C64, double kappa, double* Ti64, float* Ti32,
                  float* C32, int* status) {
  const long long nblk = 2 * nsite;
  const int grid = (int)std::min<long long>((nblk + 127) / 128, 8 * 152);
  k_clover_terms<<<grid, 128, 0, ex.stream>>>(nblk, C64, kappa, Ti64, Ti32, C32, status);
  ++*ex.launches;
}

void clover_abi(const Exec& ex, long long nsite, int L, const double* M, const cx<double>* in, cx<double>* out) {
  const long long n = nsite * L;
  k_clover_abi<<<(unsigned)((n + 255) / 256), 256, 0, ex.stream>>>(nsite, L, M, in, out);
  ++*ex.launches;
}

}  // namespace mbicg
