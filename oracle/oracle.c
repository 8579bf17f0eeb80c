/*
 * oracle.c — plain FP64 CPU oracle for arXiv:1104.0737 (Nakamura et al.,
 * "Modified Block BiCGSTAB for Lattice QCD").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the CUDA library.  It is written
 * to be checked against the paper by eye: full 4x4 spin matrices (no spin
 * projection), the steps of Algorithm 1 in the paper's order and notation,
 * modified Gram-Schmidt for the QR, LU with partial pivoting for the L x L
 * solves, and every operator applied through its plain definition.  Loops over sites are OpenMP parallel;
 * every sum is formed in a fixed order so results do not depend on the thread
 * count.
 *
 * Readings of the paper taken here:
 *  - (A phi)_x = phi_x - kappa eta_x per site (the printed sum over x in
 *    Sec. 2.1 is read as "for every x").
 *  - the backward link in Eq. (hoppingterm) is U_mu(x - mu)^dagger.
 *  - gamma basis: chiral (header), boundary: antiperiodic in t.
 *  - the WHILE condition of Algorithm 1 is read as "while max_i > eps".
 *  - M_SAP = K sum_{j=0}^{ncycle-1} (1 - A K)^j: ncycle applications of K.
 *  - B_EE, B_OO: nmr minimal-residual steps per domain and per column.
 *  - gamma of the QR is discarded; R~ = R_0 unless given.
 *  - Sec. 2.2 SSOR: L_EE = kappa T^{-1} x (hops to x + mu inside the domain),
 *    U_EE the same for x - mu; N_SSOR is the upper limit of the printed sum.
 *  - clover: T = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} F_{mu nu},
 *    F = (Q - Q^dagger)/8 over the four same-sense plaquettes; the Jacobi-
 *    preconditioned matrix is A = T^{-1} (T - kappa H).
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define NCHUNK 64 /* fixed number of partial sums for every reduction */

/* ------------------------------------------------------------------------ */
/* Gamma matrices, chiral basis.                                             */
/* ------------------------------------------------------------------------ */
static void gamma_matrices(cplx g[4][4][4]) {
  memset(g, 0, sizeof(cplx) * 64);
  /* gamma_1: off-diagonal blocks -i sigma_1 (upper right), +i sigma_1 (lower left) */
  g[0][0][3] = -I; g[0][1][2] = -I; g[0][2][1] = I; g[0][3][0] = I;
  /* gamma_2: -i sigma_2 = [[0,-1],[1,0]], +i sigma_2 = [[0,1],[-1,0]] */
  g[1][0][3] = -1; g[1][1][2] = 1; g[1][2][1] = 1; g[1][3][0] = -1;
  /* gamma_3: -i sigma_3 = diag(-i, i), +i sigma_3 = diag(i, -i) */
  g[2][0][2] = -I; g[2][1][3] = I; g[2][2][0] = I; g[2][3][1] = -I;
  /* gamma_4: identity off-diagonal blocks */
  g[3][0][2] = 1; g[3][1][3] = 1; g[3][2][0] = 1; g[3][3][1] = 1;
}

void oracle_gamma(double* out) {
  cplx g[4][4][4];
  gamma_matrices(g);
  memcpy(out, g, sizeof(g));
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
static long volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], long s, int c[4]) {
  c[0] = (int)(s % d[0]); s /= d[0];
  c[1] = (int)(s % d[1]); s /= d[1];
  c[2] = (int)(s % d[2]); s /= d[2];
  c[3] = (int)s;
}

static long site_index(const int d[4], const int c[4]) {
  return c[0] + (long)d[0] * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3]));
}

/* Neighbour of site c in direction mu, dir = +1 or -1.  *phase is -1 when the
 * hop crosses the time boundary (antiperiodic in t), +1 otherwise. */
static long neighbour(const int d[4], const int c[4], int mu, int dir, double* phase) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  *phase = 1.0;
  n[mu] += dir;
  if (n[mu] == d[mu]) { n[mu] = 0; if (mu == 3) *phase = -1.0; }
  if (n[mu] < 0) { n[mu] = d[mu] - 1; if (mu == 3) *phase = -1.0; }
  return site_index(d, n);
}

static int valid_dims(const int d[4]) {
  for (int mu = 0; mu < 4; ++mu) if (d[mu] < 1) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Wilson-Dirac operator, Sec. 2.1                                           */
/* ------------------------------------------------------------------------ */
int oracle_apply_D(const int dims[4], const double* Ud, double kappa,
                   const double* ind, double* outd, int L) {
  if (!valid_dims(dims) || L < 1 || !Ud || !ind || !outd || ind == outd) return -1;
  const cplx* U = (const cplx*)Ud;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
  const long V = volume(dims);
  cplx g[4][4][4];
  gamma_matrices(g);
  const long site_len = 12L * L; /* complex numbers per site */

#pragma omp parallel
  {
    cplx* eta = (cplx*)malloc(sizeof(cplx) * site_len);
    cplx* w = (cplx*)malloc(sizeof(cplx) * site_len);
#pragma omp for schedule(static)
    for (long s = 0; s < V; ++s) {
      int c[4];
      coords(dims, s, c);
      for (long k = 0; k < site_len; ++k) eta[k] = 0;
      for (int mu = 0; mu < 4; ++mu) {
        for (int dir = +1; dir >= -1; dir -= 2) {
          double ph;
          const long nb = neighbour(dims, c, mu, dir, &ph);
          const cplx* phin = in + nb * site_len;
          /* colour part: w = U_mu(x) phi_{x+mu} (forward) or
           * U_mu(x-mu)^dagger phi_{x-mu} (backward), times the boundary phase */
          const cplx* Ulink = (dir > 0) ? U + (s * 4 + mu) * 9 : U + (nb * 4 + mu) * 9;
          for (int sp = 0; sp < 4; ++sp)
            for (int a = 0; a < 3; ++a)
              for (int i = 0; i < L; ++i) {
                cplx acc = 0;
                for (int b = 0; b < 3; ++b) {
                  const cplx u = (dir > 0) ? Ulink[a * 3 + b] : conj(Ulink[b * 3 + a]);
                  acc += u * phin[(sp * 3 + b) * L + i];
                }
                w[(sp * 3 + a) * L + i] = ph * acc;
              }
          /* spin part: (1 - gamma_mu) forward, (1 + gamma_mu) backward */
          const double sgn = (dir > 0) ? -1.0 : 1.0;
          for (int sp = 0; sp < 4; ++sp)
            for (int t = 0; t < 4; ++t) {
              const cplx m = (sp == t ? 1.0 : 0.0) + sgn * g[mu][sp][t];
              if (m == 0) continue;
              for (int a = 0; a < 3; ++a)
                for (int i = 0; i < L; ++i)
                  eta[(sp * 3 + a) * L + i] += m * w[(t * 3 + a) * L + i];
            }
        }
      }
      const cplx* phis = in + s * site_len;
      cplx* o = out + s * site_len;
      for (long k = 0; k < site_len; ++k) o[k] = phis[k] - kappa * eta[k];
    }
    free(eta);
    free(w);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reductions and block algebra (N x L blocks, rhs index fastest)            */
/* ------------------------------------------------------------------------ */

/* out[i][j] = sum_n conj(A[n][i]) B[n][j]  (L x L, row major) */
static void block_gram(const cplx* A, const cplx* B, long N, int L, cplx* out) {
  cplx* part = (cplx*)calloc((size_t)NCHUNK * L * L, sizeof(cplx));
#pragma omp parallel for schedule(static)
  for (int ch = 0; ch < NCHUNK; ++ch) {
    const long n0 = N * ch / NCHUNK, n1 = N * (ch + 1) / NCHUNK;
    cplx* p = part + (long)ch * L * L;
    for (long n = n0; n < n1; ++n)
      for (int i = 0; i < L; ++i) {
        const cplx a = conj(A[n * L + i]);
        for (int j = 0; j < L; ++j) p[i * L + j] += a * B[n * L + j];
      }
  }
  for (int k = 0; k < L * L; ++k) out[k] = 0;
  for (int ch = 0; ch < NCHUNK; ++ch)
    for (int k = 0; k < L * L; ++k) out[k] += part[(long)ch * L * L + k];
  free(part);
}

/* Y = X M  (X: N x L, M: L x L).  Y may not alias X. */
static void block_times(const cplx* X, const cplx* M, long N, int L, cplx* Y) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n)
    for (int j = 0; j < L; ++j) {
      cplx acc = 0;
      for (int k = 0; k < L; ++k) acc += X[n * L + k] * M[k * L + j];
      Y[n * L + j] = acc;
    }
}

/* column norms |x_i| */
static void column_norms(const cplx* X, long N, int L, double* out) {
  double* part = (double*)calloc((size_t)NCHUNK * L, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int ch = 0; ch < NCHUNK; ++ch) {
    const long n0 = N * ch / NCHUNK, n1 = N * (ch + 1) / NCHUNK;
    for (long n = n0; n < n1; ++n)
      for (int i = 0; i < L; ++i) {
        const cplx v = X[n * L + i];
        part[ch * L + i] += creal(v) * creal(v) + cimag(v) * cimag(v);
      }
  }
  for (int i = 0; i < L; ++i) {
    double s = 0;
    for (int ch = 0; ch < NCHUNK; ++ch) s += part[ch * L + i];
    out[i] = sqrt(s);
  }
  free(part);
}

/* ------------------------------------------------------------------------ */
/* QR by modified Gram-Schmidt, Sec. 2.1                                     */
/* ------------------------------------------------------------------------ */

/* sum_n conj(A[n][i]) A[n][j] for one pair of columns, fixed-order partials */
static cplx column_dot(const cplx* A, long N, int L, int i, int j) {
  cplx part[NCHUNK];
#pragma omp parallel for schedule(static)
  for (int ch = 0; ch < NCHUNK; ++ch) {
    const long n0 = N * ch / NCHUNK, n1 = N * (ch + 1) / NCHUNK;
    cplx s = 0;
    for (long n = n0; n < n1; ++n) s += conj(A[n * L + i]) * A[n * L + j];
    part[ch] = s;
  }
  cplx s = 0;
  for (int ch = 0; ch < NCHUNK; ++ch) s += part[ch];
  return s;
}

int oracle_qr_mgs(double* Pd, long N, int L, double* gammad) {
  if (!Pd || N < 1 || L < 1) return -1;
  cplx* P = (cplx*)Pd;
  cplx* gm = (cplx*)gammad;
  if (gm) for (int k = 0; k < L * L; ++k) gm[k] = 0;
  for (int j = 0; j < L; ++j) {
    /* subtract the projections on the columns already orthonormalised */
    for (int i = 0; i < j; ++i) {
      const cplx r = column_dot(P, N, L, i, j);
      if (gm) gm[i * L + j] = r;
#pragma omp parallel for schedule(static)
      for (long n = 0; n < N; ++n) P[n * L + j] -= r * P[n * L + i];
    }
    const double nrm = sqrt(creal(column_dot(P, N, L, j, j)));
    if (!(nrm > 0.0)) return 2;
    if (gm) gm[j * L + j] = nrm;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) P[n * L + j] /= nrm;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* L x L solves: LU with partial pivoting                                    */
/* ------------------------------------------------------------------------ */
int oracle_lu_solve(const double* Gd, double* Cd, int L, int M) {
  if (!Gd || !Cd || L < 1 || M < 1) return -1;
  cplx* A = (cplx*)malloc(sizeof(cplx) * L * L);
  memcpy(A, Gd, sizeof(cplx) * L * L);
  cplx* C = (cplx*)Cd;
  int status = 0;
  for (int k = 0; k < L; ++k) {
    int piv = k;
    double best = cabs(A[k * L + k]);
    for (int r = k + 1; r < L; ++r)
      if (cabs(A[r * L + k]) > best) { best = cabs(A[r * L + k]); piv = r; }
    if (!(best > 0.0)) { status = 2; break; }
    if (piv != k) {
      for (int c = 0; c < L; ++c) { cplx t = A[k * L + c]; A[k * L + c] = A[piv * L + c]; A[piv * L + c] = t; }
      for (int c = 0; c < M; ++c) { cplx t = C[k * M + c]; C[k * M + c] = C[piv * M + c]; C[piv * M + c] = t; }
    }
    for (int r = k + 1; r < L; ++r) {
      const cplx f = A[r * L + k] / A[k * L + k];
      A[r * L + k] = 0;
      for (int c = k + 1; c < L; ++c) A[r * L + c] -= f * A[k * L + c];
      for (int c = 0; c < M; ++c) C[r * M + c] -= f * C[k * M + c];
    }
  }
  if (status == 0) {
    for (int k = L - 1; k >= 0; --k)
      for (int c = 0; c < M; ++c) {
        cplx s = C[k * M + c];
        for (int j = k + 1; j < L; ++j) s -= A[k * L + j] * C[j * M + c];
        C[k * M + c] = s / A[k * L + k];
      }
  }
  free(A);
  return status;
}

/* ------------------------------------------------------------------------ */
/* SAP preconditioner, Sec. 2.2                                              */
/* ------------------------------------------------------------------------ */
static int domain_of(const int d[4], const int blk[4], const int c[4], int* colour) {
  int b[4], nb[4];
  for (int mu = 0; mu < 4; ++mu) { b[mu] = c[mu] / blk[mu]; nb[mu] = d[mu] / blk[mu]; }
  *colour = (b[0] + b[1] + b[2] + b[3]) & 1;
  return b[0] + nb[0] * (b[1] + nb[1] * (b[2] + nb[2] * b[3]));
}

int oracle_domain_colour(const int dims[4], const int block[4], int s) {
  int c[4], colour;
  coords(dims, s, c);
  domain_of(dims, block, c, &colour);
  return colour;
}

static int valid_blocking(const int d[4], const int blk[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    if (blk[mu] < 1 || d[mu] % blk[mu] != 0) return 0;
    const int nd = d[mu] / blk[mu];
    if (nd < 2 || nd % 2 != 0) return 0;
  }
  return 1;
}

/* zero every site that is not in a domain of colour `colour` */
static void mask_colour(const int d[4], const int blk[4], int colour, cplx* v, int L) {
  const long V = volume(d);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    int c[4], col;
    coords(d, s, c);
    domain_of(d, blk, c, &col);
    if (col != colour)
      for (long k = 0; k < 12L * L; ++k) v[s * 12L * L + k] = 0;
  }
}

/* M_SAP with MR domain solves for the matrix A of oracle_apply_A (A = D when
 * Tinvd is NULL). */
static int sap_mr(const int dims[4], const int block[4], const double* Ud, double kappa,
                  const double* Tinvd, int ncycle, int nmr, int mr_mode, double* omega_table,
                  const double* etad, double* psid, int L) {
  if (!valid_dims(dims) || !valid_blocking(dims, block) || ncycle < 0 || nmr < 0 || L < 1)
    return -1;
  if (mr_mode < 0 || mr_mode > 2 || (mr_mode == 2 && !omega_table)) return -1;
  cplx* table = (cplx*)omega_table;
  const cplx* eta = (const cplx*)etad;
  cplx* psi = (cplx*)psid;
  const long V = volume(dims);
  const long NL = 12L * V * L;
  int nd = 1;
  for (int mu = 0; mu < 4; ++mu) nd *= dims[mu] / block[mu];
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * NL);
  cplx* r = (cplx*)malloc(sizeof(cplx) * NL);
  cplx* x = (cplx*)malloc(sizeof(cplx) * NL);
  cplx* q = (cplx*)malloc(sizeof(cplx) * NL);
  cplx* num = (cplx*)malloc(sizeof(cplx) * nd * L);
  double* den = (double*)malloc(sizeof(double) * nd * L);
  int* dom = (int*)malloc(sizeof(int) * V);
  int* col = (int*)malloc(sizeof(int) * V);
  for (long s = 0; s < V; ++s) {
    int c[4];
    coords(dims, s, c);
    dom[s] = domain_of(dims, block, c, &col[s]);
  }
  /* sites of each domain, in increasing site order */
  long* dstart = (long*)calloc((size_t)nd + 1, sizeof(long));
  long* dsites = (long*)malloc(sizeof(long) * V);
  for (long s = 0; s < V; ++s) dstart[dom[s] + 1]++;
  for (int dd = 0; dd < nd; ++dd) dstart[dd + 1] += dstart[dd];
  {
    long* fill = (long*)malloc(sizeof(long) * nd);
    for (int dd = 0; dd < nd; ++dd) fill[dd] = dstart[dd];
    for (long s = 0; s < V; ++s) dsites[fill[dom[s]]++] = s;
    free(fill);
  }

  for (long k = 0; k < NL; ++k) psi[k] = 0;
  for (int cyc = 0; cyc < ncycle; ++cyc) {
    for (int colour = 0; colour < 2; ++colour) {
      /* current residual rho = eta - A psi, restricted to the colour */
      oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)psi, (double*)tmp, L);
#pragma omp parallel for schedule(static)
      for (long k = 0; k < NL; ++k) { r[k] = eta[k] - tmp[k]; x[k] = 0; }
      mask_colour(dims, block, colour, r, L);
      /* nmr minimal-residual steps on every domain of this colour:
       * q = A_cc r (the colour-diagonal block of A, i.e. the domain operators
       * with Dirichlet boundaries), omega = (q^H r)/(q^H q), x += omega r,
       * r -= omega q, one omega per domain and per column */
      for (int it = 0; it < nmr; ++it) {
        oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)r, (double*)q, L);
        mask_colour(dims, block, colour, q, L);
#pragma omp parallel for schedule(dynamic)
        for (int dd = 0; dd < nd; ++dd) {
          for (int i = 0; i < L; ++i) { num[(long)dd * L + i] = 0; den[(long)dd * L + i] = 0; }
          for (long m = dstart[dd]; m < dstart[dd + 1]; ++m) {
            const long s = dsites[m];
            if (col[s] != colour) continue;
            for (int sc = 0; sc < 12; ++sc)
              for (int i = 0; i < L; ++i) {
                const long k = (s * 12 + sc) * L + i;
                num[(long)dd * L + i] += conj(q[k]) * r[k];
                den[(long)dd * L + i] += creal(q[k]) * creal(q[k]) + cimag(q[k]) * cimag(q[k]);
              }
          }
        }
        /* step lengths: per column (mode 0), shared by the columns of the
         * block (mode 1, the sums over columns), or frozen (mode 2): a table
         * entry is recorded from the block sums the first time its domain's
         * MR residual is nonzero and reused from then on.  Where the residual
         * is exactly zero the step length multiplies zero, so every call is
         * the same linear operator, the one of the final table. */
        for (int dd = 0; dd < nd; ++dd) {
          cplx* tab = table ? table + (((long)cyc * 2 + colour) * nmr + it) * nd + dd : NULL;
          if (mr_mode == 0) {
            for (int i = 0; i < L; ++i) {
              const long di = (long)dd * L + i;
              num[di] = den[di] > 0 ? num[di] / den[di] : 0;
            }
          } else {
            cplx om;
            if (mr_mode == 2 && !isnan(creal(*tab))) {
              om = *tab;
            } else {
              cplx n_sum = 0;
              double d_sum = 0;
              for (int i = 0; i < L; ++i) { n_sum += num[(long)dd * L + i]; d_sum += den[(long)dd * L + i]; }
              om = d_sum > 0 ? n_sum / d_sum : 0;
              if (mr_mode == 2 && d_sum > 0) *tab = om;
            }
            for (int i = 0; i < L; ++i) num[(long)dd * L + i] = om;
          }
        }
#pragma omp parallel for schedule(static)
        for (long s = 0; s < V; ++s) {
          if (col[s] != colour) continue;
          for (int sc = 0; sc < 12; ++sc)
            for (int i = 0; i < L; ++i) {
              const long k = (s * 12 + sc) * L + i;
              const cplx om = num[(long)dom[s] * L + i];
              x[k] += om * r[k];
              r[k] -= om * q[k];
            }
        }
      }
#pragma omp parallel for schedule(static)
      for (long k = 0; k < NL; ++k) psi[k] += x[k];
    }
  }
  free(tmp); free(r); free(x); free(q); free(num); free(den); free(dom); free(col);
  free(dstart); free(dsites);
  return 0;
}

int oracle_sap(const int dims[4], const int block[4], const double* Ud, double kappa,
               int ncycle, int nmr, int mr_mode, double* omega_table,
               const double* etad, double* psid, int L) {
  return sap_mr(dims, block, Ud, kappa, NULL, ncycle, nmr, mr_mode, omega_table, etad, psid, L);
}

/* ------------------------------------------------------------------------ */
/* Clover term and Jacobi preconditioning, Sec. 2.2                          */
/* ------------------------------------------------------------------------ */
/* out = a b for 3x3 colour matrices, each factor optionally daggered */
static void mat3_mul(const cplx* a, int dag_a, const cplx* b, int dag_b, cplx* out) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) {
        const cplx x = dag_a ? conj(a[k * 3 + i]) : a[i * 3 + k];
        const cplx y = dag_b ? conj(b[j * 3 + k]) : b[k * 3 + j];
        acc += x * y;
      }
      out[i * 3 + j] = acc;
    }
}

/* site c + dm mu + dn nu, periodic (links carry no boundary phase) */
static long site_plus(const int d[4], const int c[4], int mu, int dm, int nu, int dn) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  n[mu] = ((n[mu] + dm) % d[mu] + d[mu]) % d[mu];
  n[nu] = ((n[nu] + dn) % d[nu] + d[nu]) % d[nu];
  return site_index(d, n);
}

/* ordered product of four links l[0] l[1] l[2] l[3], l[k] daggered if dag[k] */
static void loop4(const cplx* const l[4], const int dag[4], cplx* out) {
  cplx t1[9], t2[9];
  mat3_mul(l[0], dag[0], l[1], dag[1], t1);
  mat3_mul(t1, 0, l[2], dag[2], t2);
  mat3_mul(t2, 0, l[3], dag[3], out);
}

int oracle_clover(const int dims[4], const double* Ud, double kappa, double csw, double* Td) {
  if (!valid_dims(dims) || !Ud || !Td) return -1;
  const cplx* U = (const cplx*)Ud;
  cplx* T = (cplx*)Td;
  const long V = volume(dims);
  cplx g[4][4][4];
  gamma_matrices(g);
  /* sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] */
  cplx sigma[4][4][4][4];
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          cplx comm = 0;
          for (int k = 0; k < 4; ++k) comm += g[mu][r][k] * g[nu][k][c] - g[nu][r][k] * g[mu][k][c];
          sigma[mu][nu][r][c] = 0.5 * I * comm;
        }
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    int c[4];
    coords(dims, s, c);
    cplx* Ts = T + s * 144;
    for (int k = 0; k < 144; ++k) Ts[k] = 0;
    for (int k = 0; k < 12; ++k) Ts[k * 12 + k] = 1;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) {
        /* the four plaquettes of the (mu, nu) plane at x, each traversed
         * mu before nu: right-up-left-down, up-left-down-right,
         * left-down-right-up, down-right-up-left */
        const long xp = site_plus(dims, c, mu, 1, nu, 0), xn = site_plus(dims, c, mu, 0, nu, 1);
        const long xm = site_plus(dims, c, mu, -1, nu, 0), xmn = site_plus(dims, c, mu, -1, nu, -1);
        const long xd = site_plus(dims, c, mu, 0, nu, -1), xpd = site_plus(dims, c, mu, 1, nu, -1);
        const long xmu = site_plus(dims, c, mu, -1, nu, 1);
        const cplx* l1[4] = {U + (s * 4 + mu) * 9, U + (xp * 4 + nu) * 9, U + (xn * 4 + mu) * 9, U + (s * 4 + nu) * 9};
        const int d1[4] = {0, 0, 1, 1};
        const cplx* l2[4] = {U + (s * 4 + nu) * 9, U + (xmu * 4 + mu) * 9, U + (xm * 4 + nu) * 9, U + (xm * 4 + mu) * 9};
        const int d2[4] = {0, 1, 1, 0};
        const cplx* l3[4] = {U + (xm * 4 + mu) * 9, U + (xmn * 4 + nu) * 9, U + (xmn * 4 + mu) * 9, U + (xd * 4 + nu) * 9};
        const int d3[4] = {1, 1, 0, 0};
        const cplx* l4[4] = {U + (xd * 4 + nu) * 9, U + (xd * 4 + mu) * 9, U + (xpd * 4 + nu) * 9, U + (s * 4 + mu) * 9};
        const int d4[4] = {1, 0, 0, 1};
        cplx Q[9] = {0}, w[9];
        loop4(l1, d1, w); for (int k = 0; k < 9; ++k) Q[k] += w[k];
        loop4(l2, d2, w); for (int k = 0; k < 9; ++k) Q[k] += w[k];
        loop4(l3, d3, w); for (int k = 0; k < 9; ++k) Q[k] += w[k];
        loop4(l4, d4, w); for (int k = 0; k < 9; ++k) Q[k] += w[k];
        /* F = (Q - Q^dagger) / 8;  T += i kappa csw sigma_{mu nu} (x) F */
        cplx F[9];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) F[a * 3 + b] = (Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0;
        for (int r = 0; r < 4; ++r)
          for (int cc = 0; cc < 4; ++cc) {
            const cplx sg = sigma[mu][nu][r][cc];
            if (sg == 0) continue;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                Ts[(r * 3 + a) * 12 + cc * 3 + b] += I * kappa * csw * sg * F[a * 3 + b];
          }
      }
  }
  return 0;
}

int oracle_clover_inverse(long V, const double* Td, double* Tinvd) {
  if (V < 1 || !Td || !Tinvd || Td == Tinvd) return -1;
  const cplx* T = (const cplx*)Td;
  cplx* Ti = (cplx*)Tinvd;
  int status = 0;
#pragma omp parallel for schedule(static) reduction(max : status)
  for (long s = 0; s < V; ++s) {
    cplx* X = Ti + s * 144;
    for (int k = 0; k < 144; ++k) X[k] = 0;
    for (int k = 0; k < 12; ++k) X[k * 12 + k] = 1;
    const int rc = oracle_lu_solve((const double*)(T + s * 144), (double*)X, 12, 12);
    if (rc != 0) status = 2;
  }
  return status;
}

/* out (12 L) = M in (12 L) for a 12 x 12 spin-colour matrix M at one site */
static void site_matrix_apply(const cplx* M, const cplx* in, int L, cplx* out) {
  for (int r = 0; r < 12; ++r)
    for (int i = 0; i < L; ++i) {
      cplx acc = 0;
      for (int c = 0; c < 12; ++c) acc += M[r * 12 + c] * in[c * L + i];
      out[r * L + i] = acc;
    }
}

/* The hopping term of Eq. (hoppingterm) (Sec. 2.1) at one site s, split by
 * direction:
 *   which & 1   forward   sum_mu (1 - gamma_mu) U_mu(x) v_{x+mu}
 *   which & 2   backward  sum_mu (1 + gamma_mu) U_mu(x-mu)^dagger v_{x-mu}
 * each hop times its boundary phase.  With dom != NULL only neighbours in the
 * same domain as s contribute (Dirichlet domain boundaries).  out: the 12 L
 * numbers of site s; w: 12 L scratch. */
static void hop_site(const int d[4], const cplx* U, const cplx g[4][4][4], const int* dom,
                     long s, int which, const cplx* v, int L, cplx* out, cplx* w) {
  int c[4];
  coords(d, s, c);
  for (long k = 0; k < 12L * L; ++k) out[k] = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int dir = +1; dir >= -1; dir -= 2) {
      if (!(which & (dir > 0 ? 1 : 2))) continue;
      double ph;
      const long nb = neighbour(d, c, mu, dir, &ph);
      if (dom && dom[nb] != dom[s]) continue;
      const cplx* vn = v + nb * 12L * L;
      const cplx* Ul = (dir > 0) ? U + (s * 4 + mu) * 9 : U + (nb * 4 + mu) * 9;
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a)
          for (int i = 0; i < L; ++i) {
            cplx acc = 0;
            for (int b = 0; b < 3; ++b) {
              const cplx u = (dir > 0) ? Ul[a * 3 + b] : conj(Ul[b * 3 + a]);
              acc += u * vn[(sp * 3 + b) * L + i];
            }
            w[(sp * 3 + a) * L + i] = ph * acc;
          }
      const double sgn = (dir > 0) ? -1.0 : 1.0;
      for (int sp = 0; sp < 4; ++sp)
        for (int t = 0; t < 4; ++t) {
          const cplx m = (sp == t ? 1.0 : 0.0) + sgn * g[mu][sp][t];
          if (m == 0) continue;
          for (int a = 0; a < 3; ++a)
            for (int i = 0; i < L; ++i) out[(sp * 3 + a) * L + i] += m * w[(t * 3 + a) * L + i];
        }
    }
}

int oracle_apply_clover_D(const int dims[4], const double* Ud, double kappa, const double* Td,
                          const double* ind, double* outd, int L) {
  if (!valid_dims(dims) || L < 1 || !Ud || !Td || !ind || !outd || ind == outd) return -1;
  const cplx* U = (const cplx*)Ud;
  const cplx* T = (const cplx*)Td;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
  const long V = volume(dims);
  cplx g[4][4][4];
  gamma_matrices(g);
#pragma omp parallel
  {
    cplx* eta = (cplx*)malloc(sizeof(cplx) * 12 * L);
    cplx* w = (cplx*)malloc(sizeof(cplx) * 12 * L);
    cplx* tp = (cplx*)malloc(sizeof(cplx) * 12 * L);
#pragma omp for schedule(static)
    for (long s = 0; s < V; ++s) {
      hop_site(dims, U, g, NULL, s, 3, in, L, eta, w);
      site_matrix_apply(T + s * 144, in + s * 12L * L, L, tp);
      for (long k = 0; k < 12L * L; ++k) out[s * 12L * L + k] = tp[k] - kappa * eta[k];
    }
    free(eta); free(w); free(tp);
  }
  return 0;
}

int oracle_apply_A(const int dims[4], const double* Ud, double kappa, const double* Tinvd,
                   const double* ind, double* outd, int L) {
  if (!Tinvd) return oracle_apply_D(dims, Ud, kappa, ind, outd, L);
  if (!valid_dims(dims) || L < 1 || !Ud || !ind || !outd || ind == outd) return -1;
  const cplx* U = (const cplx*)Ud;
  const cplx* Ti = (const cplx*)Tinvd;
  const cplx* in = (const cplx*)ind;
  cplx* out = (cplx*)outd;
  const long V = volume(dims);
  cplx g[4][4][4];
  gamma_matrices(g);
#pragma omp parallel
  {
    cplx* eta = (cplx*)malloc(sizeof(cplx) * 12 * L);
    cplx* w = (cplx*)malloc(sizeof(cplx) * 12 * L);
    cplx* h = (cplx*)malloc(sizeof(cplx) * 12 * L);
#pragma omp for schedule(static)
    for (long s = 0; s < V; ++s) {
      hop_site(dims, U, g, NULL, s, 3, in, L, eta, w);
      site_matrix_apply(Ti + s * 144, eta, L, h);
      for (long k = 0; k < 12L * L; ++k) out[s * 12L * L + k] = in[s * 12L * L + k] - kappa * h[k];
    }
    free(eta); free(w); free(h);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* SSOR domain solves, Sec. 2.2                                              */
/* ------------------------------------------------------------------------ */
/* A = 1 - L - U on a domain with L = kappa T^{-1} (forward hops inside the
 * domain) and U = kappa T^{-1} (backward hops inside the domain); T = 1 for
 * the Wilson matrix.  A forward hop reaches a larger site index and a
 * backward hop a smaller one (no domain wraps around the lattice), so L is
 * strictly triangular in decreasing site order and U in increasing order. */
typedef struct {
  const int* d;
  const cplx* U;
  const cplx* Tinv;        /* NULL: T = 1 */
  const cplx (*g)[4][4];
  const int* dom;          /* domain of every site */
  double kappa, omega;
  int L;
} ssor_ctx;

/* z = (1 - omega L)^{-1} y (which = 1) or z = (1 - omega U)^{-1} y (which = 2)
 * on the sites of one domain (sites[0..n-1] in increasing order), by
 * substitution: z_x = y_x + omega kappa T_x^{-1} (hops of z)_x */
static void ssor_triangular(const ssor_ctx* c, const long* sites, long n, int which,
                            const cplx* y, cplx* z, cplx* h, cplx* w, cplx* th) {
  const long len = 12L * c->L;
  for (long m = 0; m < n; ++m) {
    const long s = sites[which == 1 ? n - 1 - m : m];
    hop_site(c->d, c->U, c->g, c->dom, s, which, z, c->L, h, w);
    const cplx* hh = h;
    if (c->Tinv) { site_matrix_apply(c->Tinv + s * 144, h, c->L, th); hh = th; }
    for (long k = 0; k < len; ++k) z[s * len + k] = y[s * len + k] + c->omega * c->kappa * hh[k];
  }
}

/* out = B y on one domain (Sec. 2.2, the SSOR approximation of the inverse of
 * the domain matrix):
 *   B = (1 - omega U)^{-1} [sum_{j=0}^{nssor} (1 - Ahat)^j] (1 - omega L)^{-1},
 *   Ahat = (1/omega) [(1 - omega L)^{-1} + (1 - omega U)^{-1}
 *                     + (omega - 2) (1 - omega L)^{-1} (1 - omega U)^{-1}].
 * work: 6 full-lattice blocks (only this domain's sites are touched). */
static void ssor_domain(const ssor_ctx* c, const long* sites, long n, int nssor,
                        const cplx* y, cplx* out, cplx* const work[6], cplx* h, cplx* w, cplx* th) {
  const long len = 12L * c->L;
  cplx *p = work[0], *acc = work[1], *term = work[2], *qv = work[3], *pv = work[4], *pqv = work[5];
  ssor_triangular(c, sites, n, 1, y, p, h, w, th);
  for (long m = 0; m < n; ++m)
    for (long k = 0; k < len; ++k) {
      const long e = sites[m] * len + k;
      acc[e] = p[e];
      term[e] = p[e];
    }
  for (int j = 1; j <= nssor; ++j) {
    ssor_triangular(c, sites, n, 2, term, qv, h, w, th);  /* (1 - omega U)^{-1} term */
    ssor_triangular(c, sites, n, 1, term, pv, h, w, th);  /* (1 - omega L)^{-1} term */
    ssor_triangular(c, sites, n, 1, qv, pqv, h, w, th);   /* (1 - omega L)^{-1} (1 - omega U)^{-1} term */
    for (long m = 0; m < n; ++m)
      for (long k = 0; k < len; ++k) {
        const long e = sites[m] * len + k;
        const cplx ahat = (pv[e] + qv[e] + (c->omega - 2.0) * pqv[e]) / c->omega;
        term[e] -= ahat;
        acc[e] += term[e];
      }
  }
  ssor_triangular(c, sites, n, 2, acc, out, h, w, th);
}

typedef struct {
  int nd;
  int* dom;      /* domain of each site */
  int* col;      /* colour of each site */
  long* dstart;  /* sites of domain k: dsites[dstart[k] .. dstart[k+1]-1], increasing */
  long* dsites;
} domain_lists;

static void domain_lists_make(const int d[4], const int blk[4], domain_lists* dl) {
  const long V = volume(d);
  dl->nd = 1;
  for (int mu = 0; mu < 4; ++mu) dl->nd *= d[mu] / blk[mu];
  dl->dom = (int*)malloc(sizeof(int) * V);
  dl->col = (int*)malloc(sizeof(int) * V);
  dl->dstart = (long*)calloc((size_t)dl->nd + 1, sizeof(long));
  dl->dsites = (long*)malloc(sizeof(long) * V);
  for (long s = 0; s < V; ++s) {
    int c[4];
    coords(d, s, c);
    dl->dom[s] = domain_of(d, blk, c, &dl->col[s]);
    dl->dstart[dl->dom[s] + 1]++;
  }
  for (int k = 0; k < dl->nd; ++k) dl->dstart[k + 1] += dl->dstart[k];
  long* fill = (long*)malloc(sizeof(long) * dl->nd);
  for (int k = 0; k < dl->nd; ++k) fill[k] = dl->dstart[k];
  for (long s = 0; s < V; ++s) dl->dsites[fill[dl->dom[s]]++] = s;
  free(fill);
}

static void domain_lists_free(domain_lists* dl) {
  free(dl->dom); free(dl->col); free(dl->dstart); free(dl->dsites);
}

/* out = B_cc in: the SSOR domain solve on every domain of colour `colour`
 * (the domains of one colour are independent); out is zero on the other
 * colour.  work: 6 full-lattice blocks. */
static void ssor_colour(const ssor_ctx* c, const domain_lists* dl, int colour, int nssor,
                        const cplx* in, cplx* out, cplx* const work[6], long NL) {
  for (long k = 0; k < NL; ++k) out[k] = 0;
#pragma omp parallel
  {
    cplx* h = (cplx*)malloc(sizeof(cplx) * 12 * c->L);
    cplx* w = (cplx*)malloc(sizeof(cplx) * 12 * c->L);
    cplx* th = (cplx*)malloc(sizeof(cplx) * 12 * c->L);
#pragma omp for schedule(dynamic)
    for (int k = 0; k < dl->nd; ++k) {
      const long* sites = dl->dsites + dl->dstart[k];
      const long n = dl->dstart[k + 1] - dl->dstart[k];
      if (n == 0 || dl->col[sites[0]] != colour) continue;
      ssor_domain(c, sites, n, nssor, in, out, work, h, w, th);
    }
    free(h); free(w); free(th);
  }
}

int oracle_ssor_domains(const int dims[4], const int block[4], const double* Ud, double kappa,
                        const double* Tinvd, int nssor, double omega, int colour,
                        const double* ind, double* outd, int L) {
  if (!valid_dims(dims) || !valid_blocking(dims, block) || L < 1 || nssor < 0) return -1;
  if (!(omega > 0.0 && omega < 2.0) || (colour != 0 && colour != 1) || !Ud || !ind || !outd ||
      ind == outd)
    return -1;
  const long NL = 12L * volume(dims) * L;
  cplx g[4][4][4];
  gamma_matrices(g);
  domain_lists dl;
  domain_lists_make(dims, block, &dl);
  ssor_ctx c = {dims, (const cplx*)Ud, (const cplx*)Tinvd, (const cplx(*)[4][4])g, dl.dom, kappa, omega, L};
  cplx* work[6];
  for (int k = 0; k < 6; ++k) work[k] = (cplx*)calloc((size_t)NL, sizeof(cplx));
  ssor_colour(&c, &dl, colour, nssor, (const cplx*)ind, (cplx*)outd, work, NL);
  for (int k = 0; k < 6; ++k) free(work[k]);
  domain_lists_free(&dl);
  return 0;
}

/* M_SAP with SSOR domain solves (Sec. 2.2): ncycle applications of K, each an
 * E sweep then an O sweep on the updated residual, for the matrix A of
 * oracle_apply_A. */
static int sap_ssor(const int dims[4], const int block[4], const double* Ud, double kappa,
                    const double* Tinvd, int ncycle, int nssor, double omega,
                    const double* etad, double* psid, int L) {
  const cplx* eta = (const cplx*)etad;
  cplx* psi = (cplx*)psid;
  const long NL = 12L * volume(dims) * L;
  cplx g[4][4][4];
  gamma_matrices(g);
  domain_lists dl;
  domain_lists_make(dims, block, &dl);
  ssor_ctx c = {dims, (const cplx*)Ud, (const cplx*)Tinvd, (const cplx(*)[4][4])g, dl.dom, kappa, omega, L};
  cplx* work[6];
  for (int k = 0; k < 6; ++k) work[k] = (cplx*)calloc((size_t)NL, sizeof(cplx));
  cplx* r = (cplx*)malloc(sizeof(cplx) * NL);
  cplx* delta = (cplx*)malloc(sizeof(cplx) * NL);
  for (long k = 0; k < NL; ++k) psi[k] = 0;
  for (int cyc = 0; cyc < ncycle; ++cyc)
    for (int colour = 0; colour < 2; ++colour) {
      /* residual rho = eta - A psi; the domain solves read only this colour */
      oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)psi, (double*)r, L);
      for (long k = 0; k < NL; ++k) r[k] = eta[k] - r[k];
      ssor_colour(&c, &dl, colour, nssor, r, delta, work, NL);
      for (long k = 0; k < NL; ++k) psi[k] += delta[k];
    }
  for (int k = 0; k < 6; ++k) free(work[k]);
  free(r); free(delta);
  domain_lists_free(&dl);
  return 0;
}

int oracle_sap_ext(const int dims[4], const int block[4], const double* U, double kappa,
                   const double* Tinv, int ncycle, int solver, int nmr, int mr_mode,
                   double* omega_table, int nssor, double omega,
                   const double* eta, double* psi, int L) {
  if (solver == ORACLE_DOMAIN_MR)
    return sap_mr(dims, block, U, kappa, Tinv, ncycle, nmr, mr_mode, omega_table, eta, psi, L);
  if (solver != ORACLE_DOMAIN_SSOR) return -1;
  if (!valid_dims(dims) || !valid_blocking(dims, block) || ncycle < 0 || nssor < 0 || L < 1 ||
      !(omega > 0.0 && omega < 2.0) || !U || !eta || !psi || eta == psi)
    return -1;
  return sap_ssor(dims, block, U, kappa, Tinv, ncycle, nssor, omega, eta, psi, L);
}

/* ------------------------------------------------------------------------ */
/* Modified block BiCGSTAB, Algorithm 1                                      */
/* ------------------------------------------------------------------------ */
/* M = M_SAP, or M = 1 when ncycle == 0; with MR domain solves in mr_mode 2
 * one table of frozen step lengths serves every application in the solve. */
typedef struct {
  const int* block;
  const double* Tinv;
  int ncycle, solver, nmr, mr_mode, nssor;
  double omega;
  double* table;
} precond;

static void apply_M(const int dims[4], const double* U, double kappa, const precond* pc,
                    const cplx* in, cplx* out, int L, long NL) {
  if (pc->ncycle == 0) {
    memcpy(out, in, sizeof(cplx) * NL);
  } else {
    oracle_sap_ext(dims, pc->block, U, kappa, pc->Tinv, pc->ncycle, pc->solver, pc->nmr,
                   pc->mr_mode, pc->table, pc->nssor, pc->omega, (const double*)in, (double*)out, L);
  }
}

static double max_rel(const double* rn, const double* bn, int L) {
  double m = 0;
  for (int i = 0; i < L; ++i) {
    const double v = rn[i] / bn[i];
    if (!(v <= m)) m = v; /* propagates NaN */
  }
  return m;
}

int oracle_block_bicgstab_ext(const int dims[4], const double* Ud, double kappa,
                              const double* Tinvd, const double* Bd, double* Xd, int L,
                              double tol, int max_iter, int use_x0, const double* rtilde,
                              int ncycle, int solver, int nmr, int mr_mode, int nssor,
                              double omega, const int block[4], double* history,
                              int history_len, int* iters, double* true_res) {
  if (!valid_dims(dims) || L < 1 || !(tol > 0) || max_iter < 0) return -1;
  if (ncycle > 0 && (!block || !valid_blocking(dims, block))) return -1;
  if (mr_mode < 0 || mr_mode > 2) return -1;
  if (solver != ORACLE_DOMAIN_MR && solver != ORACLE_DOMAIN_SSOR) return -1;
  if (ncycle > 0 && solver == ORACLE_DOMAIN_SSOR && (nssor < 0 || !(omega > 0.0 && omega < 2.0)))
    return -1;
  double* table = NULL;
  if (ncycle > 0 && solver == ORACLE_DOMAIN_MR && mr_mode == 2) {
    long nd = 1;
    for (int mu = 0; mu < 4; ++mu) nd *= dims[mu] / block[mu];
    const long n = 2L * ncycle * 2 * (nmr > 0 ? nmr : 1) * nd;
    table = (double*)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) table[i] = NAN; /* every entry unrecorded */
  }
  const precond pc = {block, Tinvd, ncycle, solver, nmr, mr_mode, nssor, omega, table};
  const long N = 12L * volume(dims);
  const long NL = N * L;
  const cplx* B = (const cplx*)Bd;
  cplx* X = (cplx*)Xd;
  cplx *R = malloc(sizeof(cplx) * NL), *P = malloc(sizeof(cplx) * NL),
       *Rt = malloc(sizeof(cplx) * NL), *Ub = malloc(sizeof(cplx) * NL),
       *Vb = malloc(sizeof(cplx) * NL), *T = malloc(sizeof(cplx) * NL),
       *S = malloc(sizeof(cplx) * NL), *Z = malloc(sizeof(cplx) * NL),
       *W = malloc(sizeof(cplx) * NL);
  cplx *G = malloc(sizeof(cplx) * L * L), *alpha = malloc(sizeof(cplx) * L * L),
       *beta = malloc(sizeof(cplx) * L * L);
  double *bn = malloc(sizeof(double) * L), *rn = malloc(sizeof(double) * L);
  int status = 0, k = 0;

  column_norms(B, N, L, bn);
  for (int i = 0; i < L; ++i)
    if (!(bn[i] > 0)) { status = -1; goto done; }

  /* the initial guess */
  if (!use_x0) memset(X, 0, sizeof(cplx) * NL);
  /* R = B - A X */
  oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)X, (double*)W, L);
  for (long n = 0; n < NL; ++n) R[n] = B[n] - W[n];
  /* P = R */
  memcpy(P, R, sizeof(cplx) * NL);
  /* R~: the caller's, else R */
  if (rtilde) memcpy(Rt, rtilde, sizeof(cplx) * NL);
  else memcpy(Rt, R, sizeof(cplx) * NL);

  column_norms(R, N, L, rn);
  while (max_rel(rn, bn, L) > tol) {
    if (k >= max_iter) { status = 1; break; }
    /* QR decomposition P = Q gamma, P <- Q */
    if (oracle_qr_mgs((double*)P, N, L, NULL) != 0) { status = 2; break; }
    /* U = M P */
    apply_M(dims, Ud, kappa, &pc, P, Ub, L, NL);
    /* V = A U */
    oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)Ub, (double*)Vb, L);
    /* solve (R~^H V) alpha = R~^H R */
    block_gram(Rt, Vb, N, L, G);
    block_gram(Rt, R, N, L, alpha);
    if (oracle_lu_solve((const double*)G, (double*)alpha, L, L) != 0) { status = 2; break; }
    /* T = R - V alpha */
    block_times(Vb, alpha, N, L, W);
    for (long n = 0; n < NL; ++n) T[n] = R[n] - W[n];
    /* S = M T */
    apply_M(dims, Ud, kappa, &pc, T, S, L, NL);
    /* Z = A S */
    oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)S, (double*)Z, L);
    /* zeta = Tr(Z^H T) / Tr(Z^H Z) */
    cplx zt = 0, zz = 0;
    {
      cplx* gzt = malloc(sizeof(cplx) * L * L);
      cplx* gzz = malloc(sizeof(cplx) * L * L);
      block_gram(Z, T, N, L, gzt);
      block_gram(Z, Z, N, L, gzz);
      for (int i = 0; i < L; ++i) { zt += gzt[i * L + i]; zz += gzz[i * L + i]; }
      free(gzt);
      free(gzz);
    }
    if (!(cabs(zz) > 0)) { status = 2; break; }
    const cplx zeta = zt / zz;
    /* X <- X + U alpha + zeta S */
    block_times(Ub, alpha, N, L, W);
    for (long n = 0; n < NL; ++n) X[n] += W[n] + zeta * S[n];
    /* R = T - zeta Z */
    for (long n = 0; n < NL; ++n) R[n] = T[n] - zeta * Z[n];
    /* solve (R~^H V) beta = - R~^H Z */
    block_gram(Rt, Z, N, L, beta);
    for (int q = 0; q < L * L; ++q) beta[q] = -beta[q];
    if (oracle_lu_solve((const double*)G, (double*)beta, L, L) != 0) { status = 2; break; }
    /* P <- R + (P - zeta V) beta */
    for (long n = 0; n < NL; ++n) T[n] = P[n] - zeta * Vb[n];
    block_times(T, beta, N, L, W);
    for (long n = 0; n < NL; ++n) P[n] = R[n] + W[n];

    column_norms(R, N, L, rn);
    if (history && k < history_len) history[k] = max_rel(rn, bn, L);
    ++k;
  }

  /* true residual |b_i - A x_i| / |b_i| */
  oracle_apply_A(dims, Ud, kappa, Tinvd, (const double*)X, (double*)W, L);
  for (long n = 0; n < NL; ++n) W[n] = B[n] - W[n];
  column_norms(W, N, L, rn);
  if (true_res)
    for (int i = 0; i < L; ++i) true_res[i] = rn[i] / bn[i];

done:
  if (iters) *iters = k;
  free(R); free(P); free(Rt); free(Ub); free(Vb); free(T); free(S); free(Z); free(W);
  free(G); free(alpha); free(beta); free(bn); free(rn);
  free(table);
  return status;
}

int oracle_block_bicgstab(const int dims[4], const double* Ud, double kappa,
                          const double* Bd, double* Xd, int L, double tol, int max_iter,
                          int use_x0, const double* rtilde,
                          int ncycle, int nmr, int mr_mode, const int block[4],
                          double* history, int history_len, int* iters, double* true_res) {
  return oracle_block_bicgstab_ext(dims, Ud, kappa, NULL, Bd, Xd, L, tol, max_iter, use_x0,
                                   rtilde, ncycle, ORACLE_DOMAIN_MR, nmr, mr_mode, 0, 0.0,
                                   block, history, history_len, iters, true_res);
}
