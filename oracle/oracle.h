/*
 * oracle.h — plain FP64 CPU oracle for the Wilson-Dirac block solve of
 * Nakamura, Ishikawa, Kuramashi, Sakurai, Tadano, "Modified Block BiCGSTAB for
 * Lattice QCD" (arXiv:1104.0737).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (all arrays interleaved complex128, caller owned):
 *   site   s = x + Lx*(y + Ly*(z + Lz*t)),   dims = {Lx, Ly, Lz, Lt}
 *   links  U[s][mu][a][b]                    mu = 0..3 for x, y, z, t;
 *          U_mu(x) is the link from x to x+mu, no boundary phase folded in
 *   block  psi[s][spin 4][colour 3][rhs L]   the right-hand-side index runs
 *          fastest, as in Sec. 2.1 (the i = 1..L loop innermost)
 * Boundary conditions: periodic in x, y, z; antiperiodic in t (a hop across
 * the t wrap carries a factor -1).
 * Gamma matrices: Hermitian chiral basis,
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1, 2, 3),
 *   gamma_4 = [[0, 1], [1, 0]],   gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
 *
 * Return codes: 0 ok, 1 not converged within max_iter, 2 breakdown
 * (a zero pivot in the QR or in the L x L solve), -1 bad arguments.
 */
#ifndef MBICG_ORACLE_H
#define MBICG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Copies the four 4x4 gamma matrices (gamma_1..gamma_4) into g[mu][row][col]
 * as interleaved complex (2*64 doubles). */
void oracle_gamma(double* g);

/* out = A in, with (A phi)_x = phi_x - kappa * eta_x and eta_x the hopping term
 * of Eq. (hoppingterm) of Sec. 2.1, applied column by column (Eq.
 * (bloclhoppingterm)).  in and out must not alias. */
int oracle_apply_D(const int dims[4], const double* U, double kappa,
                   const double* in, double* out, int L);

/* Domain colour of site s for SAP domains of extent block[4]: the parity of
 * the sum of the domain coordinates (0 = even "E", 1 = odd "O"). */
int oracle_domain_colour(const int dims[4], const int block[4], int s);

/* psi = M_SAP eta, Sec. 2.2: ncycle applications of the multiplicative Schwarz
 * step K (E domains, then O domains on the updated residual), i.e.
 * psi = K sum_{j=0}^{ncycle-1} (1 - A K)^j eta.  The domain solves B_EE, B_OO
 * are nmr steps of minimal residual on each domain, started from zero.  The
 * complex step lengths omega = (q^H r)/(q^H q) are
 *   mr_mode 0: one per domain and per column;
 *   mr_mode 1: one per domain, from the sums of q^H r and q^H q over the L
 *              columns;
 *   mr_mode 2: frozen: one per domain taken from omega_table; an entry that is
 *              NaN (unrecorded) is recorded from the mode-1 sums the first
 *              time that domain's residual is nonzero.  With one table shared
 *              by several calls, every call applies the same linear operator.
 * omega_table: complex [ncycle][2 colours][nmr][domain] (mode 2 only), domain
 * numbered lexicographically over domain coordinates (x fastest).
 * Every extent of block must divide dims and give an even number (>= 2) of
 * domains per direction. */
int oracle_sap(const int dims[4], const int block[4], const double* U, double kappa,
               int ncycle, int nmr, int mr_mode, double* omega_table,
               const double* eta, double* psi, int L);

/* QR decomposition of an N x L block by modified Gram-Schmidt (Sec. 2.1):
 * P = Q gamma with gamma upper triangular with real positive diagonal.
 * On return P holds Q; gamma (L x L, row major, complex) is written if not NULL.
 * Returns 2 if a column becomes zero. */
int oracle_qr_mgs(double* P, long N, int L, double* gamma);

/* Solves G X = C for X (L x L complex G, L x M complex C, row major) by LU
 * decomposition with partial pivoting.  C is overwritten by X.  Returns 2 on a
 * zero pivot. */
int oracle_lu_solve(const double* G, double* C, int L, int M);

/* Modified block BiCGSTAB, Algorithm 1 (Sec. 2.1), right-preconditioned with
 * M = M_SAP (ncycle, nmr, block) or M = 1 when ncycle == 0.  mr_mode as in
 * oracle_sap; with mr_mode 2 one table of frozen step lengths (all entries
 * unrecorded at the start) serves every application of M in the solve, so M
 * is one fixed linear operator (the stationary preconditioner Sec. 2.1 asks
 * for).
 *   B, X       N x L blocks in the layout above; X is the initial guess when
 *               use_x0 != 0, otherwise it is set to zero first.
 *   rtilde      the shadow block R~; NULL selects R~ = R_0.
 *   tol         stop when max_i |r_i| / |b_i| <= tol (recursive residual).
 *   history     if not NULL, history[k] = max_i |r_i|/|b_i| after iteration k
 *               (k = 0 .. max_iter-1); history_len entries at most.
 *   iters       iterations done.
 *   true_res    L entries, |b_i - A x_i| / |b_i| at return.
 */
int oracle_block_bicgstab(const int dims[4], const double* U, double kappa,
                          const double* B, double* X, int L, double tol, int max_iter,
                          int use_x0, const double* rtilde,
                          int ncycle, int nmr, int mr_mode, const int block[4],
                          double* history, int history_len, int* iters, double* true_res);

/* ---- Sec. 2.2: the O(a)-improved operator, Jacobi preconditioning, SSOR ---- */

/* The site-local clover matrix T_x = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
 * of the O(a)-improved Wilson-Dirac matrix D_c = T - kappa H, with
 *   sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],
 *   F_{mu nu}(x)  = (Q_{mu nu}(x) - Q_{mu nu}(x)^dagger) / 8,
 *   Q_{mu nu}(x)  = the sum of the four plaquettes of the (mu, nu) plane that
 *                   start and end at x, each traversed in the mu-then-nu sense
 *                   (no trace subtracted, no boundary phase: links only).
 * T: [site][12][12] complex, row and column index spin * 3 + colour. */
int oracle_clover(const int dims[4], const double* U, double kappa, double csw, double* T);

/* Tinv[s] = T[s]^{-1} for V sites (LU with partial pivoting per site).
 * Returns 2 if a site matrix is singular. */
int oracle_clover_inverse(long V, const double* T, double* Tinv);

/* out = D_c in = T in - kappa H in (H the hopping term of Sec. 2.1). */
int oracle_apply_clover_D(const int dims[4], const double* U, double kappa, const double* T,
                          const double* in, double* out, int L);

/* out = A in for the Jacobi-preconditioned matrix A = T^{-1} D_c
 * = 1 - kappa T^{-1} H (Sec. 2.2, the division by 1 + clover term).
 * Tinv == NULL gives the Wilson matrix (oracle_apply_D). */
int oracle_apply_A(const int dims[4], const double* U, double kappa, const double* Tinv,
                   const double* in, double* out, int L);

/* Domain solvers of the SAP preconditioner. */
#define ORACLE_DOMAIN_MR 0   /* nmr minimal-residual steps (mr_mode as in oracle_sap) */
#define ORACLE_DOMAIN_SSOR 1 /* the SSOR approximation of Sec. 2.2 */

/* out = B_cc in on every domain of colour `colour` (0 = E, 1 = O), zero on the
 * other colour, with the SSOR approximation of Sec. 2.2: on a domain with
 * matrix A_dom = 1 - L - U, L = kappa T^{-1} (forward hops inside the domain),
 * U = kappa T^{-1} (backward hops inside the domain),
 *   B = (1 - omega U)^{-1} [sum_{j=0}^{nssor} (1 - Ahat)^j] (1 - omega L)^{-1},
 *   Ahat = (1/omega) [(1 - omega L)^{-1} + (1 - omega U)^{-1}
 *                     + (omega - 2) (1 - omega L)^{-1} (1 - omega U)^{-1}],
 * the triangular inverses by substitution over the domain's sites (decreasing
 * site order for L, increasing for U).  nssor >= 0 is the upper limit of the
 * sum, as printed; 0 < omega < 2.  Tinv == NULL: T = 1 (Wilson). */
int oracle_ssor_domains(const int dims[4], const int block[4], const double* U, double kappa,
                        const double* Tinv, int nssor, double omega, int colour,
                        const double* in, double* out, int L);

/* psi = M_SAP eta as oracle_sap, for the matrix A of oracle_apply_A and with
 * either domain solver: ORACLE_DOMAIN_MR (nmr, mr_mode, omega_table as in
 * oracle_sap) or ORACLE_DOMAIN_SSOR (nssor, omega as in oracle_ssor_domains). */
int oracle_sap_ext(const int dims[4], const int block[4], const double* U, double kappa,
                   const double* Tinv, int ncycle, int solver, int nmr, int mr_mode,
                   double* omega_table, int nssor, double omega,
                   const double* eta, double* psi, int L);

/* oracle_block_bicgstab for the matrix A of oracle_apply_A (A X = B; with a
 * clover term the caller passes T^{-1} B for D_c X = B) and the SAP domain
 * solver of oracle_sap_ext.  true_res is |b_i - A x_i| / |b_i|. */
int oracle_block_bicgstab_ext(const int dims[4], const double* U, double kappa,
                              const double* Tinv, const double* B, double* X, int L,
                              double tol, int max_iter, int use_x0, const double* rtilde,
                              int ncycle, int solver, int nmr, int mr_mode, int nssor,
                              double omega, const int block[4], double* history,
                              int history_len, int* iters, double* true_res);

/* Number of OpenMP threads the oracle runs with. */
int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
