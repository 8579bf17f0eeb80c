/*
 * oracle.c — plain FP64 CPU oracle for arXiv:1104.0737 (Nakamura et al.,
 * "Modified Block BiCGSTAB for Lattice QCD").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the CUDA library.  It is written
 * to be checked against the paper by eye: full 4x4 spin matrices (no spin
 * projection), Algorithm 1 taken line by line, modified Gram-Schmidt for the
 * QR, LU with partial pivoting for the L x L solves, and every operator
 * applied through its plain definition.  Loops over sites are OpenMP parallel;
 * every sum is formed in a fixed order so results do not depend on the thread
 * count.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *  - (A phi)_x = phi_x - kappa eta_x per site (the printed sum over x in
 *    Sec. 2.1 is read as "for every x").
 *  - the backward link in Eq. (hoppingterm) is U_mu(x - mu)^dagger.
 *  - gamma basis: chiral (header), boundary: antiperiodic in t.
 *  - the WHILE condition of Algorithm 1 is read as "while max_i > eps".
 *  - M_SAP = K sum_{j=0}^{ncycle-1} (1 - A K)^j: ncycle applications of K.
 *  - B_EE, B_OO: nmr minimal-residual steps per domain and per column.
 *  - gamma of the QR is discarded; R~ = R_0 unless given.
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

int oracle_sap(const int dims[4], const int block[4], const double* Ud, double kappa,
               int ncycle, int nmr, int mr_mode, double* omega_table,
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
      oracle_apply_D(dims, Ud, kappa, (const double*)psi, (double*)tmp, L);
#pragma omp parallel for schedule(static)
      for (long k = 0; k < NL; ++k) { r[k] = eta[k] - tmp[k]; x[k] = 0; }
      mask_colour(dims, block, colour, r, L);
      /* nmr minimal-residual steps on every domain of this colour:
       * q = A_cc r (the colour-diagonal block of A, i.e. the domain operators
       * with Dirichlet boundaries), omega = (q^H r)/(q^H q), x += omega r,
       * r -= omega q, one omega per domain and per column */
      for (int it = 0; it < nmr; ++it) {
        oracle_apply_D(dims, Ud, kappa, (const double*)r, (double*)q, L);
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

/* ------------------------------------------------------------------------ */
/* Modified block BiCGSTAB, Algorithm 1                                      */
/* ------------------------------------------------------------------------ */
/* M = M_SAP, or M = 1 when ncycle == 0; with mr_mode 2 one table of frozen
 * step lengths serves every application in the solve. */
static void apply_M(const int dims[4], const int block[4], const double* U, double kappa,
                    int ncycle, int nmr, int mr_mode, double* table,
                    const cplx* in, cplx* out, int L, long NL) {
  if (ncycle == 0) {
    memcpy(out, in, sizeof(cplx) * NL);
  } else {
    oracle_sap(dims, block, U, kappa, ncycle, nmr, mr_mode, table, (const double*)in,
               (double*)out, L);
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

int oracle_block_bicgstab(const int dims[4], const double* Ud, double kappa,
                          const double* Bd, double* Xd, int L, double tol, int max_iter,
                          int use_x0, const double* rtilde,
                          int ncycle, int nmr, int mr_mode, const int block[4],
                          double* history, int history_len, int* iters, double* true_res) {
  if (!valid_dims(dims) || L < 1 || !(tol > 0) || max_iter < 0) return -1;
  if (ncycle > 0 && (!block || !valid_blocking(dims, block))) return -1;
  if (mr_mode < 0 || mr_mode > 2) return -1;
  double* table = NULL;
  if (ncycle > 0 && mr_mode == 2) {
    long nd = 1;
    for (int mu = 0; mu < 4; ++mu) nd *= dims[mu] / block[mu];
    const long n = 2L * ncycle * 2 * (nmr > 0 ? nmr : 1) * nd;
    table = (double*)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) table[i] = NAN; /* every entry unrecorded */
  }
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

  /* line 1: initial guess */
  if (!use_x0) memset(X, 0, sizeof(cplx) * NL);
  /* line 2: R = B - A X */
  oracle_apply_D(dims, Ud, kappa, (const double*)X, (double*)W, L);
  for (long n = 0; n < NL; ++n) R[n] = B[n] - W[n];
  /* line 3: P = R */
  memcpy(P, R, sizeof(cplx) * NL);
  /* line 4: choose R~ */
  if (rtilde) memcpy(Rt, rtilde, sizeof(cplx) * NL);
  else memcpy(Rt, R, sizeof(cplx) * NL);

  column_norms(R, N, L, rn);
  while (max_rel(rn, bn, L) > tol) {
    if (k >= max_iter) { status = 1; break; }
    /* 4.1 QR decomposition P = Q gamma, P <- Q */
    if (oracle_qr_mgs((double*)P, N, L, NULL) != 0) { status = 2; break; }
    /* 4.2 U = M P */
    apply_M(dims, block, Ud, kappa, ncycle, nmr, mr_mode, table, P, Ub, L, NL);
    /* 4.3 V = A U */
    oracle_apply_D(dims, Ud, kappa, (const double*)Ub, (double*)Vb, L);
    /* 4.4 solve (R~^H V) alpha = R~^H R */
    block_gram(Rt, Vb, N, L, G);
    block_gram(Rt, R, N, L, alpha);
    if (oracle_lu_solve((const double*)G, (double*)alpha, L, L) != 0) { status = 2; break; }
    /* 4.5 T = R - V alpha */
    block_times(Vb, alpha, N, L, W);
    for (long n = 0; n < NL; ++n) T[n] = R[n] - W[n];
    /* 4.6 S = M T */
    apply_M(dims, block, Ud, kappa, ncycle, nmr, mr_mode, table, T, S, L, NL);
    /* 4.7 Z = A S */
    oracle_apply_D(dims, Ud, kappa, (const double*)S, (double*)Z, L);
    /* 4.8 zeta = Tr(Z^H T) / Tr(Z^H Z) */
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
    /* 4.9 X <- X + U alpha + zeta S */
    block_times(Ub, alpha, N, L, W);
    for (long n = 0; n < NL; ++n) X[n] += W[n] + zeta * S[n];
    /* 4.10 R = T - zeta Z */
    for (long n = 0; n < NL; ++n) R[n] = T[n] - zeta * Z[n];
    /* 4.11 solve (R~^H V) beta = - R~^H Z */
    block_gram(Rt, Z, N, L, beta);
    for (int q = 0; q < L * L; ++q) beta[q] = -beta[q];
    if (oracle_lu_solve((const double*)G, (double*)beta, L, L) != 0) { status = 2; break; }
    /* 4.12 P <- R + (P - zeta V) beta */
    for (long n = 0; n < NL; ++n) T[n] = P[n] - zeta * Vb[n];
    block_times(T, beta, N, L, W);
    for (long n = 0; n < NL; ++n) P[n] = R[n] + W[n];

    column_norms(R, N, L, rn);
    if (history && k < history_len) history[k] = max_rel(rn, bn, L);
    ++k;
  }

  /* true residual |b_i - A x_i| / |b_i| */
  oracle_apply_D(dims, Ud, kappa, (const double*)X, (double*)W, L);
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
