// internal.h — declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

struct mbicg_ctx;  // the C ABI's opaque context (api.cu)

namespace mbicg {

// Optional per-kernel timing: an event pair around every launch, collected
// into per-class totals whenever the host synchronises anyway.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  std::vector<int> cls;         // class of each pair
  std::vector<long long> nl;    // kernel launches between the two events of each pair
  size_t used = 0;
  long long first = 0;          // launch counter at the open pair's start
  double ms[16] = {0};
  long long count[16] = {0};
  void begin(cudaStream_t s, int c, long long launches_now) {
    if (!on) return;
    if (used == cls.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      ev.push_back(a);
      ev.push_back(b);
      cls.push_back(c);
      nl.push_back(0);
    }
    cls[used] = c;
    first = launches_now;
    cudaEventRecord(ev[2 * used], s);
  }
  void end(cudaStream_t s, long long launches_now) {
    if (!on) return;
    cudaEventRecord(ev[2 * used + 1], s);
    nl[used] = launches_now - first;
    ++used;
  }
  // call after the stream has been synchronised
  void collect() {
    for (size_t i = 0; i < used; ++i) {
      float t = 0;
      if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) ms[cls[i]] += t;
      count[cls[i]] += nl[i];
    }
    used = 0;
  }
  void reset() {
    used = 0;
    for (int c = 0; c < 16; ++c) { ms[c] = 0; count[c] = 0; }
  }
  void release() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    cls.clear();
    used = 0;
  }
};

// kernel classes (same numbering as mbicg_kernel_class)
enum : int { KC_DSLASH = 0, KC_DSLASH64, KC_SAP_RESID, KC_SAP_DOMAIN, KC_SAP_UPDATE, KC_GRAM, KC_AXPY,
             KC_SMALL, KC_CONVERT, KC_SAP_SWEEP, KC_NCLASS };

// Where and how a kernel is launched; every launcher adds to *launches and
// times the launch when prof->on.
struct Exec {
  cudaStream_t stream;
  long long* launches;
  Prof* prof;
};

// RAII: time the launches in a scope as one class
struct Timed {
  const Exec& ex;
  Timed(const Exec& e, int c) : ex(e) { if (ex.prof) ex.prof->begin(ex.stream, c, *ex.launches); }
  ~Timed() { if (ex.prof) ex.prof->end(ex.stream, *ex.launches); }
};

// ---------------------------------------------------------------------------
// Wilson-Dirac operator (dslash.cu), Sec. 2.1
// ---------------------------------------------------------------------------
// out = in - kappa * H in on every site, L columns.  links12 (FP32, optional):
// the links as their first two rows, [site][mu][6] complex, 48 bytes each
// (SU(3) fields only): the FP32 Wilson operator then reads those.
// With clov != NULL: cm = 1 the Jacobi-preconditioned clover matrix
// out = in - kappa T^{-1} H in (clov = T^{-1}), cm = 2 the clover matrix
// out = in + kappa C in - kappa H in (clov = C); packed per site (herm_off).
template <typename R>
void dslash_full(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* in, cx<R>* out,
                 int L, double kappa, const R* clov = nullptr, int cm = 0, const cx<float>* links12 = nullptr);
// Times the operator's launch configurations for this lattice, L and
// precision once per process (in -> out, both overwritten-safe scratch for
// out) and records the fastest for dslash_full; does nothing while the stream
// is being captured or when the choice is already known.
template <typename R>
void tune_dslash(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* in, cx<R>* out, int L,
                 double kappa, const cx<float>* links12 = nullptr);
// the autotuner is on when MBICG_AUTOTUNE is set and not "0"
bool autotune_enabled();

// Clover term (clover.cu), Sec. 2.2: C = i c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}
// per site from the FP64 links (packed, 72 doubles per site); for one kappa
// T^{-1} = (1 + kappa C)^{-1} in FP64 and FP32 and C in FP32 (bit 0 of *status
// set if a block is singular); out = M in for a packed M on an ABI-layout
// FP64 block (in and out may alias).
void clover_field(const Exec& ex, const Geom& g, const cx<double>* U64, double csw, double* C64);
void clover_terms(const Exec& ex, long long nsite, const double* C64, double kappa, double* Ti64, float* Ti32,
                  float* C32, int* status);
void clover_abi(const Exec& ex, long long nsite, int L, const double* M, const cx<double>* in, cx<double>* out);

// ABI blocks with dummy columns: the L columns of in into the first L of Lt
// columns of out, the rest seeded Gaussian random numbers (random) or zeros;
// and back, the first L of Lt columns.
void pack_dummies(const Exec& ex, long long nsite, int L, int Lt, const cx<double>* in, cx<double>* out,
                  unsigned long long seed, bool random);
void first_columns(const Exec& ex, long long nsite, int Lt, int L, const cx<double>* in, cx<double>* out);

// the CUDA stream a context orders its work on (api.cu)
cudaStream_t ctx_stream(const ::mbicg_ctx* c);
// device bytes of the context's workspaces (its gauge copies excluded), and
// their release (after the context's stream has drained); api.cu
size_t ctx_workspace_bytes(const ::mbicg_ctx* c);
void ctx_release_workspace(::mbicg_ctx* c);

// FP16 storage (half.cu): spinor blocks q[site][rhs][12] __half2 with one FP32
// scale per (site, rhs) (the largest |re|, |im| of the spinor; the value is
// q * s), links as their first two rows [site][mu][6] __half2.
void abi_to_half(const Exec& ex, long long nsite, int L, const cx<double>* in, __half2* q, float* sc);
void half_to_abi(const Exec& ex, long long nsite, int L, const __half2* q, const float* sc, cx<double>* out);
void links_to_half(const Exec& ex, long long nsite, const cx<double>* in, __half2* l16);
// an FP32 internal block of nspinor (site, rhs) spinors <-> FP16 storage
void block_to_half(const Exec& ex, long long nspinor, const cx<float>* in, __half2* q, float* sc);
void half_to_block(const Exec& ex, long long nspinor, const __half2* q, const float* sc, cx<float>* out);
// out = in - kappa * hops with FP16 storage and FP32 arithmetic (SU(3) links)
void dslash_half(const Exec& ex, const Geom& g, const __half2* l16, const __half2* q, const float* sc, __half2* qo,
                 float* so, int L, double kappa);

// SAP pieces on the sites of the domains of one colour (the slot numbering of
// colour_slot_coords; arrays are full-lattice, in the internal layout).
//   r = eta - (psi - kappa H psi)   (psi_zero: r = eta)
//   (tinv != NULL: the Jacobi-preconditioned clover matrix, H -> T^{-1} H)
template <typename R>
void sap_residual(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const cx<R>* eta,
                  const cx<R>* psi, cx<R>* r, int L, double kappa, bool psi_zero, const R* tinv = nullptr,
                  int c0 = 0, int nc = 0, const cx<float>* links12 = nullptr);
//   q = r - kappa H_dom r  (hops leaving the domain dropped) and, if dots is
//   not NULL, per-CTA partial sums of q^H r and q^H q for every column:
//   dots[((k * nchunk) + chunk) * L + rhs] = {Re q^H r, Im q^H r, q^H q}
template <typename R>
void sap_domain_apply(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const cx<R>* r,
                      cx<R>* q, double* dots, int L, double kappa, int* nchunk_out, const R* tinv = nullptr);
// The rest of a colour sweep once its residual is formed (nmr MR steps from
// rin, then psi += x) in one kernel, the domain kept on chip by a
// thread-block cluster; FP32, MR modes 0 and 3,
// domain shapes 8^4 and 4^4, with T^{-1} (tinv) for the Jacobi-preconditioned
// clover matrix.  Returns false (nothing launched) otherwise.
// table: the frozen step lengths of this (cycle, colour), [nmr][nd/2] complex.
// rin: the residual of this colour's sites at entry (eta itself when
// psi_mode = 1, psi = 0 on entry and psi = x on exit; psi_mode = 2: psi += x).
// c0, nc: only the columns c0 .. c0 + nc - 1 of the L-column blocks (nc = 0:
// all L; the preconditioner acts on each column by itself in modes 0 and 3).
bool sap_sweep_fused(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const cx<float>* rin,
                     cx<float>* psi, int L, double kappa, int psi_mode, int nmr, int mode,
                     const double* table, const float* tinv = nullptr, int c0 = 0, int nc = 0);
// whether sap_sweep_fused takes this domain shape, MR mode and field
bool sap_sweep_fusable(const Geom& g, int mode);
// The same sweep on the preconditioner's FP16 storage: rin and psi as FP16
// spinors with per-(site, column) scales rsc, psc (half.cu's format), FP32
// arithmetic on chip.
bool sap_sweep_fused_h(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const __half2* rin,
                       const float* rsc, __half2* psi, float* psc, int L, double kappa, int psi_mode, int nmr,
                       int mode, const double* table, const float* tinv = nullptr, int c0 = 0, int nc = 0);
// Times the fused sweep's launch shapes (tune.h) on 8^4 domains once per
// process for this lattice, L, storage and operator (scratch blocks rin, psi
// of L columns, FP16 with scales rsc, psc when half; table: any nmr x nd/2
// complex step lengths of the right size) and records the fastest for the
// sweeps; does nothing while the stream is being captured or when the choice
// is already known.
void tune_sap_sweep(const Exec& ex, const Geom& g, const cx<float>* links, void* rin, float* rsc, void* psi,
                    float* psc, int L, double kappa, int nmr, const double* table, bool half, const float* tinv);
// r = eta - A psi on the sites of one colour, eta, psi and r in FP16 storage
void sap_residual_h(const Exec& ex, const Geom& g, int colour, const cx<float>* links, const __half2* eta,
                    const float* esc, const __half2* psi, const float* psc, __half2* r, float* rsc, int L, double kappa,
                    const float* tinv = nullptr, int c0 = 0, int nc = 0);
// SSOR (Sec. 2.2): one wavefront level of z = (1 - omega L)^{-1} y (fwd) or
// z = (1 - omega U)^{-1} y on every domain of one colour, L and U the forward
// and backward hops inside a domain (times T^{-1} with tinv); komega =
// kappa * omega; local[0..count) the local site indices of the level.
template <typename R>
void ssor_level(const Exec& ex, const Geom& g, int colour, const cx<R>* links, const R* tinv, const cx<R>* y,
                cx<R>* z, int L, double komega, const int* local, int count, bool fwd);
// Number of sites per CTA the SAP kernels use for L columns (divides Vd).
int sap_sites_per_cta(const Geom& g, int L, bool fp64);

// ---------------------------------------------------------------------------
// SAP preconditioner driver (sap.cu), Sec. 2.2
// ---------------------------------------------------------------------------
struct SapWork {
  void* psi = nullptr;    // full lattice, precision of the SAP
  void* r = nullptr;
  void* q = nullptr;
  void* x = nullptr;
  double* dots = nullptr;     // partial sums
  double* omega = nullptr;    // complex step lengths [domain-of-colour][rhs]
  const cx<float>* links12 = nullptr;  // FP32 links as two rows (SU(3) fields), else NULL
  size_t bytes_block = 0;     // size of one full-lattice block
  size_t dots_len = 0;
  int L = 0;
  bool fp64 = false;
  // SSOR domain solves: the local site indices of a domain sorted by
  // wavefront level lx + ly + lz + lt (device copy of level_host), level k at
  // [level_off[k], level_off[k + 1]); four full-lattice scratch blocks
  int* levels = nullptr;
  std::vector<int> level_host, level_off;
  void* ssor[4] = {nullptr, nullptr, nullptr, nullptr};
};

// The SAP domain solver (Sec. 2.2): nmr MR steps (the default) or SSOR with
// N_SSOR = nssor and relaxation omega.
struct SsorParams {
  int nssor;
  double omega;
};
// Fills w.level_host / w.level_off for the domain shape of g and copies the
// level table to w.levels (device, Vd ints) on the stream; w must stay alive
// until the copy has completed.
cudaError_t sap_prepare_ssor(const Geom& g, SapWork& w, cudaStream_t stream);

// The preconditioner's FP16 storage: psi = M_SAP eta with eta, psi and the
// colour residual r in FP16 storage (q, per-(site, column) scale), FP32
// arithmetic and FP32 links; the fused sweep only (sap_sweep_fusable), MR
// modes 0 (per column) and 3 (frozen replay of table).
struct SapHalf {
  __half2* eta;
  float* eta_sc;
  __half2* psi;
  float* psi_sc;
  __half2* r;
  float* r_sc;
};
void sap_apply_h(const Exec& ex, const Geom& g, const cx<float>* links, const SapHalf& h, int L, double kappa,
                 int ncycle, int nmr, int mr_mode, const double* table, const float* tinv = nullptr);

// psi = M_SAP eta.  eta and psi are full-lattice blocks in the internal
// layout and in the SAP precision (R).  mr_mode: 0 per column, 1 shared by the
// columns, 2 frozen while recording (NaN entries of table are recorded from
// the shared sums where the domain's residual is nonzero; *unset is raised if
// an entry stays unrecorded), 3 frozen replay.
// table = complex [ncycle][2][nmr][nd/2] (modes 2, 3).
// tinv != NULL: SAP for the Jacobi-preconditioned clover matrix.  ssor != NULL: SSOR domain solves
// instead of MR (nmr, mr_mode, table and unset unused; w.levels and w.ssor set).
template <typename R>
void sap_apply(const Exec& ex, const Geom& g, const cx<R>* links, const cx<R>* eta, cx<R>* psi,
               int L, double kappa, int ncycle, int nmr, int mr_mode, double* table, int* unset,
               SapWork& w, const R* tinv = nullptr, const SsorParams* ssor = nullptr);

// ---------------------------------------------------------------------------
// Block linear algebra (blas.cu)
// ---------------------------------------------------------------------------
constexpr int MAXL = 16;
constexpr int GRAM_CTAS = 2 * 152;  // fixed grid: deterministic partial sums

// Partial sums, per CTA, of
//   GRAM_G1: A^H B1 (L x L)      GRAM_G2: A^H B2 (L x L)
//   GRAM_D1: diag(B1^H B2)       GRAM_D2: diag(B1^H B1)
// part[cta][slot] complex double, slots [0, L*L) G1, [L*L, 2 L*L) G2, then L
// for D1 and L for D2 (real part).  A may be NULL when only D1/D2 are asked.
// Returns the number of CTAs used (<= GRAM_CTAS).
enum : int { GRAM_G1 = 1, GRAM_G2 = 2, GRAM_D1 = 4, GRAM_D2 = 8 };
// err: device status word; ST_TIMEOUT is OR-ed in if a bounded wait for a
// bulk copy gave up.
template <typename R>
int block_gram(const Exec& ex, long long nsite, int L, const cx<R>* A, const cx<R>* B1,
               const cx<R>* B2, int flags, double* part, int* err);
int gram_slots(int L);

// Y = X M row by row (M: L x L complex double on the device), in place allowed.
template <typename R>
void block_transform(const Exec& ex, long long nsite, int L, const cx<R>* X, const double* M, cx<R>* Y);

// R -= V alpha (alpha: L x L complex double on the device)
template <typename R>
void block_update_alpha(const Exec& ex, long long nsite, int L, const cx<R>* V, const double* alpha, cx<R>* Rv);

// X64 += U alpha + zeta S (the increment in R, accumulated in FP64); R -= zeta Z;
// P = R + (P - zeta V) beta; partial column norms of the new R into
// part[cta][L] (doubles).  Returns the CTAs used.
template <typename R>
int block_update_zeta(const Exec& ex, long long nsite, int L, const cx<R>* U, const double* alpha,
                      const cx<R>* S, const cx<R>* Z, const cx<R>* V, const double* zeta_beta, cx<R>* Rv,
                      cx<R>* P, cx<double>* X64, double* part);

// U12 = the first two rows of every FP32 link ([site][mu][6])
void links_to_rows(const Exec& ex, long long nsite, const cx<float>* U32, cx<float>* U12);
// dst (device) = src (registered host memory, its mapped device address),
// bytes a multiple of 16 and both 16-byte aligned: a copy kernel
void copy_from_mapped_host(const Exec& ex, const void* src, void* dst, size_t bytes);
// ABI layout [site][sc][rhs] complex128 <-> internal [site][rhs][sc] in R.
template <typename R>
void abi_to_internal(const Exec& ex, long long nsite, int L, const cx<double>* in, cx<R>* out);
template <typename R>
void internal_to_abi(const Exec& ex, long long nsite, int L, const cx<R>* in, cx<double>* out);
// elementwise precision change of an internal block (n complex numbers)
template <typename RI, typename RO>
void convert_block(const Exec& ex, long long n, const cx<RI>* in, cx<RO>* out);
// links: ABI FP64 -> internal FP64 copy and FP32 copy; flags NaN/Inf in *bad
// (bit 0) and links that are not SU(3) to 1e-10 (bit 1)
void convert_links(const Exec& ex, long long nsite, const cx<double>* in, cx<double>* l64,
                   cx<float>* l32, int* bad);
// out = B64 - W64 converted to R (W64 NULL: out = B64), with partial column
// norms (part[cta][L])
template <typename R>
int residual_from(const Exec& ex, long long nsite, int L, const cx<double>* B64,
                  const cx<double>* W64, cx<R>* out, double* part);
// scan an ABI-layout block for NaN/Inf and column norms^2 (part[cta][L])
int abi_check(const Exec& ex, long long n_rows, int L, const cx<double>* in, double* part, int* bad);

// ---------------------------------------------------------------------------
// L x L algebra on the device (single-CTA kernels, blas.cu)
// ---------------------------------------------------------------------------
// Device-side status bits written by the small kernels.
enum : int { ST_ALPHA_SINGULAR = 1, ST_ZZ_ZERO = 2, ST_CHOL_FAIL = 4, ST_NAN = 8, ST_TIMEOUT = 16 };

struct SmallWork {
  double* G;       // R~^H V (L x L complex), kept for the beta solve
  double* LU;      // LU factors of G
  int* piv;
  double* alpha;   // L x L complex
  double* zb;      // [zeta (complex), beta (L x L complex)]
  double* M;       // QR transform (L x L complex)
  double* norms;   // L doubles (squared column norms)
  int* status;
};

// alpha = (R~^H V)^-1 R~^H R from gram partials (slots 0 and 1)
void lxl_alpha(const Exec& ex, int L, const double* part, int nparts, SmallWork& w);
// zeta = Tr(Z^H R) / Tr(Z^H Z), beta = -(R~^H V)^-1 R~^H Z from partials of
// (A = R~, B1 = Z, D = Z, E = R)
void lxl_zeta_beta(const Exec& ex, int L, const double* part, int nparts, SmallWork& w);
// Cholesky of G = P^H P = gamma^H gamma, M = gamma^-1 (slot 0 partials)
// (rel_eps: a pivot below rel_eps * G_jj counts as a failure; shift > 0
// factors G + shift * max_j G_jj * I instead)
void lxl_cholesky_inverse(const Exec& ex, int L, const double* part, int nparts, SmallWork& w,
                          double rel_eps, double shift = 0.0);
// norms[i] = sum of partial column norms (part[cta][L], or gram slots when
// from_gram, using the |D|^2 slots)
void lxl_norms(const Exec& ex, int L, const double* part, int nparts, bool from_gram, SmallWork& w);

// Device state of the Krylov loop while the device decides Algorithm 2's
// WHILE test (a conditional node of a CUDA graph repeats the iteration):
// the host writes it before a launch and reads it when the loop stops.
struct LoopCtl {
  int it;           // iterations done
  int max_iter;
  int Lc;           // columns the stopping test covers
  int sloppy;       // FP32 Krylov vectors: stop for a reliable update
  double tol;
  double delta_ru;  // reliable update below delta_ru * rmax_ru
  double rmax_ru;
  double relmax;    // max_i |r_i| / |b_i| after the last iteration
};
// After one iteration: relmax from the column norms, history[it] = relmax,
// ++it, and the loop's condition: continue while no status bit is set, relmax
// is a number above tol, it < max_iter and no reliable update is due.
void loop_control(const Exec& ex, LoopCtl* ctl, const double* norms, const double* bnorm, const int* status,
                  double* hist, int hist_len, cudaGraphConditionalHandle h);

}  // namespace mbicg
