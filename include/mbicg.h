/*
 * mbicg.h — C ABI of the GB300 (sm_103a) library for the modified block
 * BiCGSTAB solve of the Wilson-Dirac equation with SAP preconditioning,
 * after Nakamura, Ishikawa, Kuramashi, Sakurai, Tadano, "Modified Block
 * BiCGSTAB for Lattice QCD", arXiv:1104.0737.
 *
 * The calls follow the paper's problem statement A X = B with N x L blocks
 * (Sec. 2.1).  Every call returns an mbicg_status; nothing aborts the process,
 * nothing crosses the ABI as an exception, and no kernel traps the GPU.
 *
 * Layouts (fixed; interleaved complex128, i.e. double re, double im):
 *   site     s = x + Lx*(y + Ly*(z + Lz*t)), dims = {Lx, Ly, Lz, Lt}
 *   links    U[s][mu][a][b], mu = 0..3 for x, y, z, t.  U_mu(x) is the link
 *            from x to x + mu; no boundary phase folded in.
 *   blocks   psi[s][spin 4][colour 3][rhs L]: the right-hand-side index runs
 *            fastest (Sec. 2.1, the i = 1..L loop innermost).
 * Physics conventions: periodic boundaries in x, y, z and antiperiodic in t
 * (a hop across the t boundary carries -1); Hermitian chiral gamma basis,
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]].
 *
 * Pointers: every block or link pointer may be host memory (pageable or
 * pinned) or device memory of the context's device; the library detects which
 * (cudaPointerGetAttributes).  Device pointers are used in place and the call
 * is ordered on the context's stream; host pointers are staged through device
 * buffers and the call returns after the result is back in host memory.
 * Device memory of another device is refused (MBICG_EINVAL).
 * The caller owns every pointer it passes; the library owns the context, its
 * copies of the gauge field and its workspaces.
 *
 * Threading: a context is used by one host thread at a time.
 */
#ifndef MBICG_H
#define MBICG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbicg_ctx mbicg_ctx;

typedef enum {
  MBICG_OK = 0,
  MBICG_EINVAL = -1,      /* bad argument: dims, L, tol, blocking, params */
  MBICG_ENOMEM = -2,      /* device allocation failed */
  MBICG_ENOGAUGE = -3,    /* no gauge field loaded */
  MBICG_ENOTCONV = -4,    /* max_iter reached; X, iters, true_res are filled */
  MBICG_EBREAKDOWN = -5,  /* singular R~^H V, zero Tr(Z^H Z) or rank-deficient P
                             again right after a restart from the current X, or
                             a fourth time (with FP32 Krylov vectors: also in
                             the FP64 continuation); X, iters, true_res filled */
  MBICG_ENAN = -6,        /* NaN or Inf in the input or in a residual norm */
  MBICG_ECUDA = -7        /* a CUDA runtime error; see mbicg_last_error */
} mbicg_status;

/* SAP domain solvers. */
typedef enum { MBICG_DOMAIN_MR = 0, MBICG_DOMAIN_SSOR = 1 } mbicg_domain_solver;

/* Arithmetic and storage precision of an operator. */
typedef enum { MBICG_FP64 = 0, MBICG_FP32 = 1, MBICG_FP16 = 2 } mbicg_prec;

/* How the minimal-residual step lengths of the SAP domain solves are formed. */
typedef enum {
  MBICG_MR_COLUMN = 0, /* one per domain and per column (plain MR on each column) */
  MBICG_MR_BLOCK = 1,  /* one per domain, from sums over the L columns */
  MBICG_MR_FROZEN = 2  /* block_solve only: one step length per domain, colour,
                          cycle and MR step, recorded (as MBICG_MR_BLOCK) the
                          first time that domain's MR residual is nonzero and
                          reused by every later application, so M is one fixed
                          linear operator for the whole solve (the stationary M
                          that Sec. 2.1 requires) */
} mbicg_mr_mode;

typedef struct {
  /* SAP preconditioner, Sec. 2.2: psi = K sum_{j=0}^{ncycle-1} (1 - A K)^j eta
   * over checkerboard-coloured domains of extent block[4]; the domain solves
   * B_EE, B_OO are nmr MR steps started from zero (1 <= nmr <= 256).
   * ncycle = 0 selects M = 1.
   * Each block[mu] must divide dims[mu] and give an even number >= 2 of
   * domains in every direction. */
  int ncycle;
  int nmr;
  int block[4];
  int mr_mode;      /* mbicg_mr_mode */
  int prec_sap;     /* MBICG_FP32 (default), MBICG_FP64, or MBICG_FP16: the
                       preconditioner's blocks (its input, output, residual
                       and psi) stored in HBM as FP16 spinors times one FP32
                       scale per (site, column), FP32 arithmetic and links,
                       the MR state on chip in FP32.  FP16 needs 8^4 or 4^4
                       domains, SU(3) links, the Wilson matrix, MR domain
                       solves with MBICG_MR_COLUMN or MBICG_MR_FROZEN (a
                       frozen table is recorded in FP32, then replayed in
                       FP16) and, in a block solve, prec_D = MBICG_FP32 */
  /* Krylov loop (Algorithm 2 of Sec. 2.1). */
  int prec_D;       /* operator and Krylov vectors: MBICG_FP64 (the paper's
                       double-precision outer solver) or MBICG_FP32 with FP64
                       X accumulation and reliable updates */
  int max_iter;
  int use_x0;       /* nonzero: X holds the initial guess on entry */
  double delta_ru;  /* reliable update when max_i |r_i|/|b_i| falls below
                       delta_ru times its value at the last update (FP32 only) */
  /* Optional host buffer: res_history[k] = max_i |r_i|/|b_i| (recursive)
   * after iteration k, at most res_history_len entries. */
  double* res_history;
  int res_history_len;
  /* Dummy right-hand sides (Sec. 2.1: where the single-vector solve fails to
   * converge the block solve may still converge when extra right-hand sides
   * play a supplementary role): dummy_rhs extra columns of Gaussian random
   * numbers (seeded by dummy_seed, a counter-based generator) are appended to
   * B for the solve; the stopping test, X and the true residuals cover the L
   * given columns only.  L + dummy_rhs <= 16.  Default 0. */
  int dummy_rhs;
  unsigned long long dummy_seed;
  /* Nonzero: the matrix is the Jacobi-preconditioned clover matrix
   * A = T^{-1} D_c of the clover term loaded by mbicg_load_clover (Sec. 2.2);
   * mbicg_block_solve solves D_c X = B as A X = T^{-1} B (true_res and the
   * stopping test refer to that system), mbicg_sap_precond preconditions A.
   * Default 0 (the Wilson matrix). */
  int clover;
  /* SAP domain solver (Sec. 2.2): MBICG_DOMAIN_MR (default: nmr minimal-
   * residual steps, mr_mode) or MBICG_DOMAIN_SSOR: the paper's SSOR
   * approximation B = (1 - omega U)^{-1} [sum_{j=0}^{nssor} (1 - A^SSOR)^j]
   * (1 - omega L)^{-1} on each domain (L, U the forward and backward hops
   * inside the domain), a fixed linear operator.  0 <= nssor <= 16,
   * 0 < ssor_omega < 2; defaults 1 and 1.26 (the paper's values). */
  int domain_solver;
  int nssor;
  double ssor_omega;
} mbicg_params;

/* Counters of the last call on a context. */
typedef struct {
  int iters;              /* Krylov iterations of the last solve */
  int reliable_updates;   /* true-residual recomputations inside the loop */
  int restarts;           /* restarts after a breakdown */
  long long kernel_launches; /* kernels the library launched during the last call */
  double true_res_max;    /* max_i |b_i - A x_i| / |b_i| at return (FP64) */
  int graph_iterations;   /* iterations run from captured CUDA graphs once the
                             frozen step lengths are recorded: a graph whose
                             conditional WHILE node repeats the iteration while
                             the device's own test of Algorithm 2's WHILE
                             condition holds (off with MBICG_DEVICE_LOOP=0: one
                             graph launch and one host check per iteration; no
                             graphs with MBICG_GRAPHS=0 or while profiling) */
  int precision_fallbacks; /* 1 when a solve with FP32 Krylov vectors broke down
                              after its restarts and was continued from its X
                              with FP64 Krylov vectors */
  int host_syncs;         /* times the host waited for the device to read a
                             residual norm or status during the last call:
                             once per iteration while the step lengths are
                             recorded, then once per stop of the device loop
                             (convergence, reliable update, restart, max_iter) */
} mbicg_stats;

/* Fills p with the defaults: ncycle 4, nmr 4, block {4,4,4,4},
 * MBICG_MR_FROZEN, prec_sap FP32, prec_D FP32, max_iter 1000, use_x0 0,
 * delta_ru 0.1, no history, no dummy right-hand sides, no clover term,
 * MR domain solves (nssor 1, ssor_omega 1.26 for SSOR). */
void mbicg_default_params(mbicg_params* p);

/* Creates a context for a lattice of extents dims on CUDA device `device`.
 * cuda_stream: a cudaStream_t to order work on, or NULL for a stream the
 * library creates.  Every extent must be even and >= 2, the volume at most
 * 2^27 sites.
 * Returns MBICG_EINVAL, MBICG_ECUDA or MBICG_ENOMEM on failure (*ctx = NULL). */
int mbicg_create(mbicg_ctx** ctx, const int dims[4], int device, void* cuda_stream);

/* Frees every device buffer the context holds.  NULL is accepted. */
void mbicg_destroy(mbicg_ctx* ctx);

/* Copies the gauge field U (layout above, 4 V SU(3) matrices, complex128)
 * into the library's own FP64, FP32 and FP16 copies and an FP32 copy of the
 * first two rows of each link (the FP16 copy keeps those two rows as well).
 * Sec. 2.1: the links of Eq. (hoppingterm).
 * Every link is checked for unitarity and det = 1 (to 1e-10); a field that is
 * not SU(3) is accepted, but the kernels that rebuild a link's third row from
 * its first two (the fused SAP sweep, the FP32 operator's two-row reads, FP16
 * storage) are then not used.  A loaded clover term is dropped.
 * MBICG_ENAN if U holds NaN or Inf.  After any failure the context holds no
 * field (MBICG_ENOGAUGE until a later load succeeds). */
int mbicg_load_gauge(mbicg_ctx* ctx, const double* U);

/* out = A in for L columns (Eq. (hoppingterm), (bloclhoppingterm) of
 * Sec. 2.1): (A phi)_x = phi_x - kappa eta_x.  prec: MBICG_FP64 computes in
 * FP64, MBICG_FP32 rounds `in` to FP32, computes in FP32 and widens the result.
 * MBICG_FP16 stores `in`, the result and the links in FP16 and computes in
 * FP32: each (site, column) spinor is kept as 12 complex FP16 numbers times
 * one FP32 scale (its largest |re| or |im|), each link as its first two rows
 * (the third is rebuilt), and the result is rounded into the same format
 * before it is widened; it needs SU(3) links (MBICG_EINVAL otherwise).
 * 1 <= L <= 16.  in and out must not alias. */
int mbicg_apply_D(mbicg_ctx* ctx, const double* in, double* out, int L, double kappa,
                  int prec);

/* Clover term of the O(a)-improved Wilson-Dirac matrix (Sec. 2.2; the paper
 * names the improvement, this is its standard clover-leaf form):
 *   D_c = T - kappa H,   T_x = 1 + kappa C_x,
 *   C_x = i csw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu],
 *   F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^dagger) / 8,
 * Q_{mu nu}(x) the four plaquettes of the (mu, nu) plane that start and end at
 * x, all traversed mu before nu.  Computes C from the loaded gauge field (FP64;
 * 72 doubles per site plus FP32 copies and the inverse of T for the kappa of
 * the next call: about 1.8 kB of device memory per site in all).  csw = 0
 * switches the clover term off.  Loading another gauge field switches it off
 * too.  Errors: MBICG_ENOGAUGE, MBICG_EINVAL (csw < 0 or not finite),
 * MBICG_ENOMEM, MBICG_ECUDA. */
int mbicg_load_clover(mbicg_ctx* ctx, double csw);

/* out = D_c in (jacobi = 0) or out = A in = T^{-1} D_c in (jacobi = 1), with
 * the clover term of mbicg_load_clover; layout, pointers and precision as
 * mbicg_apply_D (MBICG_FP64 or MBICG_FP32; FP16 is rejected).  T^{-1} is
 * formed for kappa when kappa changes (FP64 Gauss-Jordan per 6 x 6 chirality
 * block).  Errors: as mbicg_apply_D, and MBICG_EINVAL when no clover term is
 * loaded or 1 + kappa C is singular at some site. */
int mbicg_apply_clover(mbicg_ctx* ctx, const double* in, double* out, int L, double kappa, int prec,
                       int jacobi);

/* out = M_SAP in (Sec. 2.2) with the parameters ncycle, nmr, block, mr_mode
 * (MBICG_MR_COLUMN or MBICG_MR_BLOCK; MBICG_MR_FROZEN through
 * mbicg_sap_precond_frozen) and prec_sap of *p.  1 <= L <= 16. */
int mbicg_sap_precond(mbicg_ctx* ctx, const double* in, double* out, int L, double kappa,
                      const mbicg_params* p);

/* Length, in doubles, of the step-length table of mbicg_sap_precond_frozen
 * for the SAP parameters *p (ncycle, nmr, block) on this context's lattice:
 * 2 * ncycle * 2 * nmr * nd, nd = the number of domains. */
int mbicg_sap_table_len(const mbicg_ctx* ctx, const mbicg_params* p, long long* n_doubles);

/* out = M_SAP in (Sec. 2.2) with frozen MR step lengths: the preconditioner
 * that mbicg_block_solve applies by default (MBICG_MR_FROZEN, the stationary M
 * of Sec. 2.1), with its step-length table held by the caller.
 *   table     host array of mbicg_sap_table_len doubles: complex step lengths
 *             [cycle][colour][MR step][domain], the domain numbered
 *             lexicographically by its coordinates (b0 + nb0 (b1 + nb1 (b2 +
 *             nb2 b3)), nb = dims / block); entries of domains of the other
 *             colour are not used.  NaN marks an entry not yet recorded.
 *   complete  if not NULL: 1 on return when every entry the sweeps use is set.
 * If any used entry is NaN, the call records: such an entry is set to the
 * step length formed from the sums over all L columns the first time that
 * domain's MR residual is nonzero in this call (MBICG_MR_BLOCK's formula) and
 * written back to table; an entry whose domain residual stays zero stays NaN
 * (it multiplies zero).  Otherwise the table is replayed unchanged, in FP32 by
 * the fused on-chip sweep for 8^4 and 4^4 domains of an SU(3) field (the
 * kernel the block solve uses).  A sequence of calls starting from an all-NaN
 * table therefore builds the solver's table lazily, as mbicg_block_solve does.
 * p: MR domain solves with mr_mode = MBICG_MR_FROZEN, prec_sap FP32 or FP64.
 * Errors as mbicg_sap_precond; MBICG_EINVAL for a device-memory table. */
int mbicg_sap_precond_frozen(mbicg_ctx* ctx, const double* in, double* out, int L, double kappa,
                             const mbicg_params* p, double* table, int* complete);

/* Solves A X = B for L right-hand sides by the modified block BiCGSTAB
 * (Algorithm 2 of Sec. 2.1: QR re-orthonormalisation of P, right
 * preconditioning by M_SAP), stopping when max_i |r_i|/|b_i| <= tol for the
 * recursive residual and confirming it with the true residual in FP64.
 *   B          N x L block (N = 12 V), every column nonzero.
 *   X          N x L block: the solution on return (also on ENOTCONV and
 *              EBREAKDOWN); the initial guess on entry if p->use_x0.
 *   iters      if not NULL: iterations done.
 *   true_res   if not NULL: L host doubles, |b_i - A x_i| / |b_i| in FP64.
 * 1 <= L <= 16 (L + p->dummy_rhs <= 16); tol > 0.
 * The QR of P is shifted CholeskyQR3 (a first Cholesky pass on P^H P + s I,
 * s = 1e-13 (FP64 Krylov vectors) or 1e-5 (FP32) times max_j |p_j|^2, then two
 * plain passes; L = 1: two plain passes).  A breakdown (rank-deficient P, singular R~^H V,
 * Tr(Z^H Z) = 0) restarts from the current X (at most three times, not twice
 * in a row); with FP32 Krylov vectors a solve that still breaks down continues
 * from its X with FP64 Krylov vectors (mbicg_stats.precision_fallbacks).  Once
 * the frozen step lengths are recorded, the iterations run from one captured
 * CUDA graph on the context's stream whose conditional WHILE node repeats the
 * iteration while the device's own stopping test holds; the host steps in only
 * when that loop stops (convergence, reliable update, breakdown, max_iter).
 * Returns MBICG_OK, MBICG_ENOTCONV (max_iter reached or the final true
 * residual above tol), MBICG_EBREAKDOWN, MBICG_ENAN, or MBICG_EINVAL /
 * MBICG_ENOGAUGE / MBICG_ENOMEM / MBICG_ECUDA before or instead of a result. */
int mbicg_block_solve(mbicg_ctx* ctx, const double* B, double* X, int L, double kappa,
                      double tol, const mbicg_params* p, int* iters, double* true_res);

/* Counters of the last call (see mbicg_stats). */
int mbicg_get_stats(const mbicg_ctx* ctx, mbicg_stats* out);

/* Kernel classes of the per-kernel timing below. */
typedef enum {
  MBICG_K_DSLASH = 0,     /* block Wilson-Dirac operator, Krylov precision */
  MBICG_K_DSLASH64 = 1,   /* FP64 operator of the true residuals */
  MBICG_K_SAP_RESID = 2,  /* SAP: residual eta - A psi on one colour */
  MBICG_K_SAP_DOMAIN = 3, /* SAP: domain operator with the MR dot products */
  MBICG_K_SAP_UPDATE = 4, /* SAP: MR step lengths and updates */
  MBICG_K_GRAM = 5,       /* block inner products */
  MBICG_K_AXPY = 6,       /* block AXPYs and the QR transform */
  MBICG_K_SMALL = 7,      /* L x L algebra */
  MBICG_K_CONVERT = 8,    /* layout and precision conversions */
  MBICG_K_SAP_SWEEP = 9,  /* SAP: one whole colour sweep with the MR steps on chip */
  MBICG_K_NCLASS = 10
} mbicg_kernel_class;

/* enable != 0: from now on, time the library's kernel launches with CUDA
 * events on the context's stream, grouped in regions of one class (one event
 * pair per region; a region holds one or two launches, e.g. the MR step
 * length and update kernels of MBICG_K_SAP_UPDATE), and add them to their
 * class.  Every kernel launch of mbicg_block_solve belongs to a region.
 * enable == 0 stops timing.  Either way the totals are reset. */
int mbicg_set_profiling(mbicg_ctx* ctx, int enable);

/* Copies the totals since profiling was enabled: ms[c] milliseconds of the
 * regions of class c and launches[c] the kernel launches in them, for c < n
 * (n <= MBICG_K_NCLASS).  Either pointer may be NULL. */
int mbicg_get_profile(const mbicg_ctx* ctx, double* ms, long long* launches, int n);

/* Text of the last error on ctx ("" if none).  Valid until the next call. */
const char* mbicg_last_error(const mbicg_ctx* ctx);

/* Size of the fixed scratch array of mbicg_apply_D_noalloc, in MiB. */
#define MBICG_NOALLOC_SCRATCH_MB 32

/* out = A in in FP32, the same result as mbicg_apply_D(..., MBICG_FP32), for
 * callers that cannot allocate device memory: code running inside a
 * framework's memory pool that must not grow device memory behind the pool,
 * real-time or latency-bound loops that may not take the allocator's locks or
 * wait for it, programs whose device memory is fixed when they start.  It
 * allocates nothing and needs no context.  The paper has no counterpart to
 * this entry point.
 *   dims         lattice extents (even, >= 2)
 *   U, in, out   device pointers of the current device (cudaGetDevice) in the
 *                layouts above; in and out must not alias; U is the FP64
 *                gauge field (36 V complex numbers), in and out 12 V L each
 *   cuda_stream  a cudaStream_t or NULL; the work is ordered on it and the call
 *                returns without waiting for it
 * Its scratch is one file-scope device array of MBICG_NOALLOC_SCRATCH_MB MiB
 * per device, held by every process that loads the library until it exits:
 * the FP32 links (288 V bytes) and two FP32 blocks (96 L V bytes each), each
 * rounded up to 256 bytes, must fit in it, else MBICG_EINVAL (nothing is
 * launched).  Every call shares the array; calls that overlap on the GPU (two
 * streams, two host threads) race on it.  The first call on a device looks
 * the array's address up (cudaGetSymbolAddress) with that device current;
 * make that first call on each device before any stream capture begins.
 * Returns MBICG_EINVAL for bad arguments, host pointers or pointers of another
 * device (nothing launched), MBICG_ECUDA if a CUDA error was already pending
 * on entry (it is neither launched over nor cleared), if the lookup fails or
 * if one of its launches fails. */
int mbicg_apply_D_noalloc(const int dims[4], const double* U, const double* in, double* out, int L,
                          double kappa, void* cuda_stream);

/* Diagnostic (no counterpart in the paper): runs, in one CTA on `device`, the
 * bounded mbarrier wait that the kernels streaming blocks through shared
 * memory use, on a barrier that expects `expect_bytes` (a multiple of 16) that
 * no copy will deliver — or, with expect_bytes = 0, on one that completes by a
 * plain arrival — polling at most spin_limit times (1 <= spin_limit <= 2^24).
 * *timed_out = 1 when the wait gave up and the kernel returned with its error
 * flag set, 0 when it completed.  Nothing is copied, so giving up leaves no
 * transfer in flight; the device stays usable either way. */
int mbicg_selftest_bounded_wait(int device, int spin_limit, int expect_bytes, int* timed_out);

/* ------------------------------------------------------------------------
 * Serving: a request loop over resident gauge fields (no counterpart in the
 * paper, whose solver takes one block at a time; the method's block solve of
 * Sec. 2.1 is what packs the requests' columns together).
 *
 * Each field added to a server gets max_slots solver slots — a context with
 * its own CUDA stream and host thread, holding the field's links.  A request
 * is a source block B of 1..12 columns (ABI layout, host memory, copied at
 * submit) for one field, kappa and tol.  A free slot of the field takes the
 * oldest waiting request and packs behind it, in arrival order, the waiting
 * requests with the same kappa and tol that fit into one block of at most 12
 * columns; it solves the packed block with mbicg_block_solve (the field's
 * params) and hands each request its columns of X and of the true residuals.
 * Admission by HBM footprint: the server never holds more device memory than
 * its budget.  The slots' links are charged when a field is added; a packed
 * block is admitted only when the workspace of its block solve at its number
 * of columns fits beside everything already held (packing stops at the
 * request that would not fit); a slot keeps its workspace between solves;
 * when a slot cannot admit even its oldest request, idle slots release their
 * workspaces, and if that is not enough it waits for a running solve to
 * finish; when no solve is running, the request can never be admitted (fields
 * added after its submission took the budget) and its wait returns
 * MBICG_ENOMEM.  Requests arriving while slots or memory are busy wait; the slots
 * of different fields, and the slots of one field, solve concurrently.
 * Thread-safe: submit and wait may be called from any host threads, and a
 * field may be added while the slots of others are solving (calls adding
 * fields are taken one at a time).
 * ------------------------------------------------------------------------ */
typedef struct mbicg_server mbicg_server;

typedef struct {
  double queue_ms;    /* submit -> start of its block solve */
  double latency_ms;  /* submit -> result ready */
  double start_ms, done_ms;  /* steady-clock times of the block solve */
  int batch_columns;  /* columns of the block it was solved in */
} mbicg_request_info;

/* A server on `device` whose slots hold at most hbm_budget_gb gigabytes (1e9
 * bytes) of device memory: per slot 1152 V bytes of links and 4 MiB, per
 * admitted block solve of L columns about 12 V L (3 x 16 + 7 x 8 + 3 x 8 +
 * 3 x 16) bytes for FP32 Krylov vectors and FP32 SAP storage (FP64 ones count
 * 16 bytes per complex number; FP16 SAP storage adds 3 x 52 bytes per site
 * and column). */
int mbicg_server_create(mbicg_server** server, int device, double hbm_budget_gb);

/* Makes the gauge field U (dims, layout of mbicg_load_gauge) resident with up
 * to max_slots solver slots (as many as the budget holds the links of, at
 * least one, else MBICG_ENOMEM) solving with the parameters *p; *field_id
 * names it in submit. */
int mbicg_server_add_field(mbicg_server* server, const int dims[4], const double* U,
                           const mbicg_params* p, int max_slots, int* field_id);

/* Queues the solve of A X = B (L columns, 1 <= L <= 12, host memory, copied)
 * on field field_id; *request_id names it in wait.  MBICG_EINVAL for an
 * unknown field, L outside 1..12 or tol <= 0; MBICG_ENOMEM when a block of
 * this request alone could never fit in the budget beside the slots' links. */
int mbicg_server_submit(mbicg_server* server, int field_id, const double* B, int L,
                        double kappa, double tol, long long* request_id);

/* Blocks until the request is solved, then copies its columns of X (host,
 * caller owned, the request's L columns), the iterations of its block solve,
 * its true residuals (L doubles) and its timings (each may be NULL), forgets
 * the request and returns the status of its block solve (MBICG_ENOMEM, with X
 * zero, for a request that could never be admitted).  One wait per request:
 * another wait for it, while the first waits or after it returned, gets
 * MBICG_EINVAL. */
int mbicg_server_wait(mbicg_server* server, long long request_id, double* X, int* iters,
                      double* true_res, mbicg_request_info* info);

/* hold != 0: no slot starts a new block solve (solves already running
 * finish) and submitted requests wait; hold == 0 releases them, and the slots
 * form their blocks from everything waiting.  For admission control and for
 * tests that need a known packing. */
int mbicg_server_hold(mbicg_server* server, int hold);

/* Block solves run, columns solved, the widest block, solver slots. */
int mbicg_server_stats(mbicg_server* server, long long* solves, long long* columns,
                       long long* max_columns, int* slots);

/* Device memory the server holds now (links and admitted workspaces), its
 * budget, and how many times a slot had to wait for memory (each may be NULL). */
int mbicg_server_memory(mbicg_server* server, double* used_gb, double* budget_gb, long long* memory_waits);

/* Stops the slots (after their current solves) and frees everything; every
 * submitted request should have been waited for. */
void mbicg_server_destroy(mbicg_server* server);

#ifdef __cplusplus
}
#endif
#endif /* MBICG_H */
