// api.cu — the C ABI (include/mbicg.h): context, gauge field, the operator and
// preconditioner entry points, and the solver driver of Algorithm 2 (Sec. 2.1)
// in mixed precision.
//
// Solver state lives on the device for the whole solve: B and X in FP64, the
// Krylov blocks R, P, R~, U, V, S, Z in the Krylov precision T (FP64, or FP32
// with reliable updates).  The iterations run in a device-side loop (a CUDA
// graph with a conditional WHILE node): nothing leaves the device until the
// loop stops; the fallback, a graph per iteration, reads the L squared
// residual norms and a status word once per iteration for the stopping test
// of Algorithm 2.
//
// Mixed precision (FP32 Krylov loop): X accumulates in FP64; whenever
// max_i |r_i|/|b_i| has dropped by delta_ru since the last update, the true
// residual B - A X is recomputed with the FP64 operator and replaces R
// (reliable update).  Sec. 2.2 shows that sloppy right preconditioning keeps
// R = B - A X exact; the reliable updates bound the additional drift of the
// FP32 Krylov recursion.  The final answer is confirmed with the FP64 true
// residual.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mbicg.h"
#include <stdint.h>

#include "internal.h"

using namespace mbicg;

struct mbicg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int dims[4] = {0, 0, 0, 0};
  long long V = 0;
  cx<double>* U64 = nullptr;
  cx<float>* U32 = nullptr;
  __half2* U16 = nullptr;  // first two rows of each link in FP16, [site][mu][6]
  cx<float>* U12 = nullptr;  // first two rows of each FP32 link, [site][mu][6] (48 B, 16-byte aligned)
  bool gauge = false;
  bool su3 = false;  // every link SU(3): the fused SAP kernel may rebuild third rows
  std::string err;
  mbicg_stats stats{};
  long long launches = 0;
  Prof prof;
  std::map<std::string, std::pair<void*, size_t>> bufs;  // device workspaces
  double* h_small = nullptr;                            // pinned host scratch
  // clover term (clover.cu): C packed per site in FP64 and FP32, T^{-1} for
  // the kappa tinv_kappa (NaN: not formed); csw == 0: no clover term
  double csw = 0.0;
  double* C64 = nullptr;
  float* C32 = nullptr;
  double* Ti64 = nullptr;
  float* Ti32 = nullptr;
  double tinv_kappa = NAN;
};

namespace {

constexpr int H_SMALL = 4096;     // doubles of pinned host scratch
constexpr int H_CTL_IN = 2048;    // offsets (doubles) of the device loop's staging areas in it
constexpr int H_CTL_OUT = 2304;

int fail(mbicg_ctx* c, int code, const char* fmt, const char* a = "") {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, a);
  c->err = buf;
  return code;
}

int cuda_fail(mbicg_ctx* c, cudaError_t e, const char* where) {
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MBICG_ENOMEM : MBICG_ECUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);    \
  } while (0)

// device workspace by name; grows, never shrinks
int get_buf(mbicg_ctx* c, const char* name, size_t bytes, void** out) {
  auto it = c->bufs.find(name);
  if (it != c->bufs.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return MBICG_OK;
  }
  if (it != c->bufs.end()) {
    cudaFree(it->second.first);
    c->bufs.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes < 256 ? 256 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(c, e, name);
  }
  c->bufs[name] = {p, bytes};
  *out = p;
  return MBICG_OK;
}

template <typename P>
int buf(mbicg_ctx* c, const char* name, size_t count, P** out) {
  void* p = nullptr;
  const int rc = get_buf(c, name, count * sizeof(P), &p);
  *out = static_cast<P*>(p);
  return rc;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device that owns p when p is device memory (not managed memory, which
// every device may reach), else -1.
int owning_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return a.type == cudaMemoryTypeDevice ? a.device : -1;
}

// The device address of registered (page-locked, mapped) host memory, else
// NULL (pageable memory, which no kernel may read).
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

Geom lattice_geom(const mbicg_ctx* c, const int* block) {
  Geom g{};
  g.V = 1;
  g.nd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.d[mu] = c->dims[mu];
    g.V *= c->dims[mu];
    g.blk[mu] = block ? block[mu] : c->dims[mu];
    g.nb[mu] = g.d[mu] / g.blk[mu];
    g.nd *= g.nb[mu];
  }
  g.Vd = g.V / g.nd;
  g.su3 = c->su3 ? 1 : 0;
  geom_init_divisors(g);
  return g;
}

bool valid_blocking(const mbicg_ctx* c, const int* block) {
  long long vd = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (block[mu] < 1 || c->dims[mu] % block[mu] != 0) return false;
    const int nb = c->dims[mu] / block[mu];
    if (nb < 2 || nb % 2 != 0) return false;
    vd *= block[mu];
  }
  return vd <= (1 << 20);
}

Exec exec_of(mbicg_ctx* c) { return Exec{c->stream, &c->launches, &c->prof}; }

// The FP32 links as two rows for the Wilson operator when every link is
// SU(3) (the third row is rebuilt), else NULL (the full links are read).
const cx<float>* links12(const mbicg_ctx* c) { return c->su3 ? c->U12 : nullptr; }

int check_launch(mbicg_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return MBICG_OK;
}

// Host <-> device staging of an ABI block.
struct Staged {
  const void* user = nullptr;
  void* dev = nullptr;
  bool host = false;
  size_t bytes = 0;
};

int stage_in(mbicg_ctx* c, const void* user, size_t bytes, const char* name, bool copy, Staged* s) {
  s->user = user;
  s->bytes = bytes;
  s->host = !is_device_ptr(user);
  if (!s->host) {
    // the kernels read and write it directly: memory of another device would
    // be a peer access that may not be enabled
    const int d = owning_device(user);
    if (d >= 0 && d != c->device) return fail(c, MBICG_EINVAL, "%s: device memory of another device", name);
    s->dev = const_cast<void*>(user);
    return MBICG_OK;
  }
  int rc = get_buf(c, name, bytes, &s->dev);
  if (rc) return rc;
  if (copy) {
    const Exec ex = exec_of(c);
    Timed t(ex, KC_CONVERT);  // the copy is timed with the layout conversions
    // Registered host memory is read by a copy kernel over the whole grid: on
    // a GB300 (Grace host), one copy-engine transfer of a multi-GB block
    // issued after a solve ran at ~10 GB/s, ~20x below the rate of the copies
    // that followed it.
    const void* mapped = mapped_host_ptr(user);
    if (mapped && ((uintptr_t)mapped % 16) == 0 && ((uintptr_t)s->dev % 16) == 0 && bytes % 16 == 0)
      copy_from_mapped_host(ex, mapped, s->dev, bytes);
    else
      CK(cudaMemcpyAsync(s->dev, user, bytes, cudaMemcpyHostToDevice, c->stream));
  }
  return MBICG_OK;
}

int stage_out(mbicg_ctx* c, const Staged& s) {
  if (s.host) {
    {
      const Exec ex = exec_of(c);
      Timed t(ex, KC_CONVERT);
      CK(cudaMemcpyAsync(const_cast<void*>(s.user), s.dev, s.bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  return MBICG_OK;
}

// read n doubles (+ one int status) from the device through pinned memory
int read_small(mbicg_ctx* c, const double* d, int n, const int* status, double* out, int* st) {
  CK(cudaMemcpyAsync(c->h_small, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  if (status)
    CK(cudaMemcpyAsync(c->h_small + n, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  ++c->stats.host_syncs;
  memcpy(out, c->h_small, sizeof(double) * n);
  if (status) memcpy(st, c->h_small + n, sizeof(int));
  c->prof.collect();
  return MBICG_OK;
}

// column norms |b_i| of an ABI block on the device, and a NaN/Inf check
int abi_norms(mbicg_ctx* c, const cx<double>* d, int L, double* norms, bool* bad) {
  const Exec ex = exec_of(c);
  double* part;
  int* flag;
  double* nrm;
  int rc;
  if ((rc = buf(c, "abi_part", (size_t)8 * 152 * L, &part))) return rc;
  if ((rc = buf(c, "abi_flag", 1, &flag))) return rc;
  if ((rc = buf(c, "abi_norms", MAXL, &nrm))) return rc;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  int np;
  {
    Timed t(ex, KC_CONVERT);
    np = abi_check(ex, c->V * 12, L, d, part, flag);
  }
  SmallWork w{};
  w.norms = nrm;
  w.status = flag;  // lxl_norms ORs ST_NAN into it; abi_check sets bit 0
  {
    Timed t(ex, KC_SMALL);
    lxl_norms(ex, L, part, np, false, w);
  }
  if ((rc = check_launch(c, "abi_norms"))) return rc;
  int st = 0;
  if ((rc = read_small(c, nrm, L, flag, norms, &st))) return rc;
  *bad = st != 0;
  for (int i = 0; i < L; ++i) norms[i] = sqrt(norms[i]);
  return MBICG_OK;
}

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------
template <typename T>
struct Krylov {
  cx<T>*R, *P, *Rt, *U, *V, *S, *Z;
};

template <typename T, typename TS>
struct Solver {
  mbicg_ctx* c;
  Exec ex;
  Geom g;
  int L;
  double kappa;
  mbicg_params p;
  long long V;
  size_t nl;  // complex numbers per block: 12 V L
  cx<double>*B64, *X64, *W64;
  Krylov<T> k;
  cx<TS>*eta_s = nullptr, *psi_s = nullptr;  // SAP precision staging when TS != T
  SapWork sw;
  double* table = nullptr;
  int* unset = nullptr;
  bool table_complete = false;
  bool keep_table = false;  // continue with the frozen step lengths already recorded
  int Lc = 0;               // columns the stopping test covers (the others are dummies)
  SmallWork sm{};
  // Jacobi-preconditioned clover matrix: T^{-1} per site (NULL: Wilson)
  const double* ti64 = nullptr;
  const float* ti32 = nullptr;
  // the preconditioner in FP16 storage (prec_sap = MBICG_FP16, FP32 Krylov
  // vectors): its blocks once the frozen step lengths replay
  bool sap16 = false;
  SapHalf sh{};
  double *gpart, *npart;
  double h_norm[MAXL + 1];
  double bnorm[MAXL];

  const cx<T>* links_T() const;
  const cx<TS>* links_S() const;
  template <typename R>
  const R* tinv() const {
    return reinterpret_cast<const R*>(sizeof(R) == 8 ? static_cast<const void*>(ti64)
                                                     : static_cast<const void*>(ti32));
  }

  int alloc() {
    int rc;
    if ((rc = buf(c, "B64", nl, &B64))) return rc;
    if ((rc = buf(c, "X64", nl, &X64))) return rc;
    if ((rc = buf(c, "W64", nl, &W64))) return rc;
    const char* names[7] = {"kR", "kP", "kRt", "kU", "kV", "kS", "kZ"};
    cx<T>** ptrs[7] = {&k.R, &k.P, &k.Rt, &k.U, &k.V, &k.S, &k.Z};
    for (int i = 0; i < 7; ++i)
      if ((rc = buf(c, names[i], nl, ptrs[i]))) return rc;
    if (p.ncycle > 0) {
      if (!std::is_same<T, TS>::value) {
        if ((rc = buf(c, "eta_s", nl, &eta_s))) return rc;
        if ((rc = buf(c, "psi_s", nl, &psi_s))) return rc;
      }
      cx<TS>*r, *q, *x;
      if ((rc = buf(c, "sap_r", nl, &r))) return rc;
      if ((rc = buf(c, "sap_q", nl, &q))) return rc;
      if ((rc = buf(c, "sap_x", nl, &x))) return rc;
      sw.r = r;
      if (std::is_same<TS, float>::value) sw.links12 = links12(c);
      sw.q = q;
      sw.x = x;
      const int ndc = g.nd / 2;
      const int S = sap_sites_per_cta(g, L, sizeof(TS) == 8);
      const size_t nchunk = g.Vd / S;
      if ((rc = buf(c, "sap_dots", (size_t)ndc * nchunk * L * 3, &sw.dots))) return rc;
      if ((rc = buf(c, "sap_omega", (size_t)ndc * L * 2, &sw.omega))) return rc;
      if ((rc = buf(c, "sap_table", (size_t)p.ncycle * 2 * p.nmr * ndc * 2, &table))) return rc;
      if ((rc = buf(c, "sap_unset", 1, &unset))) return rc;
      if (p.domain_solver == MBICG_DOMAIN_SSOR) {
        const char* names4[4] = {"ssor_acc", "ssor_term", "ssor_pv", "ssor_pqv"};
        for (int i = 0; i < 4; ++i) {
          cx<TS>* b;
          if ((rc = buf(c, names4[i], nl, &b))) return rc;
          sw.ssor[i] = b;
        }
        if ((rc = buf(c, "ssor_levels", (size_t)g.Vd, &sw.levels))) return rc;
        CK(sap_prepare_ssor(g, sw, c->stream));
      }
      if (sap16) {
        const size_t nsp = (size_t)V * L;
        if ((rc = buf(c, "h16_eta", nl, &sh.eta)) || (rc = buf(c, "h16_eta_sc", nsp, &sh.eta_sc)) ||
            (rc = buf(c, "h16_psi", nl, &sh.psi)) || (rc = buf(c, "h16_psi_sc", nsp, &sh.psi_sc)) ||
            (rc = buf(c, "h16_r", nl, &sh.r)) || (rc = buf(c, "h16_r_sc", nsp, &sh.r_sc)))
          return rc;
      }
      // every frozen step length starts unrecorded (NaN), unless this solve
      // continues another one with the same preconditioner
      if (!keep_table)
        CK(cudaMemsetAsync(table, 0xff, sizeof(double) * (size_t)p.ncycle * 2 * p.nmr * ndc * 2, c->stream));
    }
    if ((rc = buf(c, "gpart", (size_t)GRAM_CTAS * gram_slots(L) * 2, &gpart))) return rc;
    if ((rc = buf(c, "npart", (size_t)8 * 152 * L, &npart))) return rc;
    if ((rc = buf(c, "sm_G", 2 * MAXL * MAXL, &sm.G))) return rc;
    if ((rc = buf(c, "sm_LU", 2 * MAXL * MAXL, &sm.LU))) return rc;
    if ((rc = buf(c, "sm_piv", MAXL, &sm.piv))) return rc;
    if ((rc = buf(c, "sm_alpha", 2 * MAXL * MAXL, &sm.alpha))) return rc;
    if ((rc = buf(c, "sm_zb", 2 + 2 * MAXL * MAXL, &sm.zb))) return rc;
    if ((rc = buf(c, "sm_M", 2 * MAXL * MAXL, &sm.M))) return rc;
    if ((rc = buf(c, "sm_norms", MAXL, &sm.norms))) return rc;
    if ((rc = buf(c, "sm_status", 1, &sm.status))) return rc;
    if (autotune_enabled()) {
      // the operator's launch shape, once per lattice, L and precision (before any capture)
      tune_dslash<T>(ex, g, links_T(), k.U, k.V, L, kappa, ti64 ? nullptr : links12(c));
      tune_dslash<double>(ex, g, c->U64, X64, W64, L, kappa);
      // the fused sweep's launch shape, on the SAP scratch blocks
      if (p.ncycle > 0 && std::is_same<TS, float>::value && p.domain_solver == MBICG_DOMAIN_MR &&
          sap_sweep_fusable(g, 3)) {
        if (sap16)
          tune_sap_sweep(ex, g, c->U32, sh.r, sh.r_sc, sh.psi, sh.psi_sc, L, kappa, p.nmr, table, true,
                         tinv<float>());
        else
          tune_sap_sweep(ex, g, c->U32, sw.r, nullptr, sw.q, nullptr, L, kappa, p.nmr, table, false, tinv<float>());
      }
    }
    return MBICG_OK;
  }

  // out = M in (T precision blocks)
  int apply_M(const cx<T>* in, cx<T>* out) {
    if (p.ncycle == 0) {
      CK(cudaMemcpyAsync(out, in, sizeof(cx<T>) * nl, cudaMemcpyDeviceToDevice, c->stream));
      return MBICG_OK;
    }
    const SsorParams sp{p.nssor, p.ssor_omega};
    const SsorParams* ssor = p.domain_solver == MBICG_DOMAIN_SSOR ? &sp : nullptr;
    // SSOR: a fixed linear operator, no step lengths to record
    int mode = ssor ? MBICG_MR_COLUMN : p.mr_mode;
    double* tab = nullptr;
    if (mode == MBICG_MR_FROZEN) {
      // record until every entry of the table is set, then replay only
      mode = table_complete ? 3 : 2;
      tab = table;
      if (!table_complete) CK(cudaMemsetAsync(unset, 0, sizeof(int), c->stream));
    }
    if constexpr (std::is_same<T, float>::value) {
      if (sap16 && (mode == 0 || mode == 3)) {
        // FP16 storage: P (or R) rounded into FP16 blocks, M applied on them
        // with FP32 arithmetic, the result widened into U (or S)
        {
          Timed t(ex, KC_CONVERT);
          block_to_half(ex, V * L, reinterpret_cast<const cx<float>*>(in), sh.eta, sh.eta_sc);
        }
        sap_apply_h(ex, g, c->U32, sh, L, kappa, p.ncycle, p.nmr, mode, tab, tinv<float>());
        {
          Timed t(ex, KC_CONVERT);
          half_to_block(ex, V * L, sh.psi, sh.psi_sc, reinterpret_cast<cx<float>*>(out));
        }
        return check_launch(c, "apply_M");
      }
    }
    if constexpr (std::is_same<T, TS>::value) {
      sap_apply<TS>(ex, g, links_S(), in, out, L, kappa, p.ncycle, p.nmr, mode, tab, unset, sw, tinv<TS>(), ssor);
    } else {
      {
        Timed t(ex, KC_CONVERT);
        convert_block<T, TS>(ex, (long long)nl, in, eta_s);
      }
      sap_apply<TS>(ex, g, links_S(), eta_s, psi_s, L, kappa, p.ncycle, p.nmr, mode, tab, unset, sw, tinv<TS>(),
                    ssor);
      Timed t(ex, KC_CONVERT);
      convert_block<TS, T>(ex, (long long)nl, psi_s, out);
    }
    if (mode == 2) {
      int flag = 1;
      CK(cudaMemcpyAsync(c->h_small, unset, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      ++c->stats.host_syncs;
      memcpy(&flag, c->h_small, sizeof(int));
      table_complete = (flag == 0);
    }
    return check_launch(c, "apply_M");
  }

  int dslash(const cx<T>* in, cx<T>* out) {
    Timed t(ex, KC_DSLASH);
    dslash_full<T>(ex, g, links_T(), in, out, L, kappa, tinv<T>(), ti64 ? 1 : 0, ti64 ? nullptr : links12(c));
    return MBICG_OK;
  }

  // R = B - A X in FP64, converted to T; host norms in h_norm.  x_zero: X = 0
  // is known, so R = B without applying the operator.
  int true_residual(double* rel, double* relmax, bool x_zero = false) {
    if (!x_zero) {
      Timed t(ex, KC_DSLASH64);
      dslash_full<double>(ex, g, c->U64, X64, W64, L, kappa, ti64, ti64 ? 1 : 0);
    }
    int np;
    {
      Timed t(ex, KC_CONVERT);
      np = residual_from<T>(ex, V, L, B64, x_zero ? nullptr : W64, k.R, npart);
    }
    {
      Timed t(ex, KC_SMALL);
      lxl_norms(ex, L, npart, np, false, sm);
    }
    int rc = check_launch(c, "true_residual");
    if (rc) return rc;
    int st = 0;
    if ((rc = read_small(c, sm.norms, L, sm.status, h_norm, &st))) return rc;
    *relmax = 0;
    for (int i = 0; i < L; ++i) {
      if (i == Lc) break;
      rel[i] = sqrt(h_norm[i]) / bnorm[i];
      if (!(rel[i] <= *relmax)) *relmax = rel[i];
    }
    return MBICG_OK;
  }

  // QR of P by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto,
  // Yanagisawa 2020): a first pass on P^H P + s I (s = 1e-5 max_j |p_j|^2
  // with FP32 Krylov vectors, 1e-13 max_j |p_j|^2 with FP64 ones), then two
  // plain passes.  A plain Cholesky of the Gram matrix fails once cond(P)
  // passes ~1/sqrt(u) (4e3 in FP32, 1e8 in FP64: nearly dependent right-hand
  // sides reach it without a preconditioner); the shifted pass brings any P of
  // cond up to ~1/u to a well-conditioned basis of the same space first, and
  // the plain passes then give the Q of the unique QR.  One column (L = 1) is
  // only normalised: two plain passes.
  int qr() {
    const int npass = L == 1 ? 2 : 3;
    const double shift = sizeof(T) == 4 ? 1e-5 : 1e-13;
    for (int pass = 0; pass < npass; ++pass) {
      int np;
      {
        Timed t(ex, KC_GRAM);
        np = block_gram<T>(ex, V, L, k.P, k.P, nullptr, GRAM_G1, gpart, sm.status);
      }
      {
        Timed t(ex, KC_SMALL);
        lxl_cholesky_inverse(ex, L, gpart, np, sm, sizeof(T) == 4 ? 1e-12 : 1e-26,
                             (L > 1 && pass == 0) ? shift : 0.0);
      }
      Timed t(ex, KC_AXPY);
      block_transform<T>(ex, V, L, k.P, sm.M, k.P);
    }
    return check_launch(c, "qr");
  }

  // One iteration's launches (the loop body of Algorithm 2) and the column
  // norms, with no host synchronisation (so that it can be captured).
  int iteration_launches() {
    int rc;
    // QR of P
    if ((rc = qr())) return rc;
    // U = M P, V = A U
    if ((rc = apply_M(k.P, k.U))) return rc;
    if ((rc = dslash(k.U, k.V))) return rc;
    // (R~^H V) alpha = R~^H R
    {
      int np;
      {
        Timed t(ex, KC_GRAM);
        np = block_gram<T>(ex, V, L, k.Rt, k.V, k.R, GRAM_G1 | GRAM_G2, gpart, sm.status);
      }
      Timed t(ex, KC_SMALL);
      lxl_alpha(ex, L, gpart, np, sm);
    }
    // R -= V alpha (X += U alpha is folded into the update after zeta)
    {
      Timed t(ex, KC_AXPY);
      block_update_alpha<T>(ex, V, L, k.V, sm.alpha, k.R);
    }
    // S = M R, Z = A S
    if ((rc = apply_M(k.R, k.S))) return rc;
    if ((rc = dslash(k.S, k.Z))) return rc;
    // zeta = Tr(Z^H R)/Tr(Z^H Z), (R~^H V) beta = -R~^H Z
    {
      int np;
      {
        Timed t(ex, KC_GRAM);
        np = block_gram<T>(ex, V, L, k.Rt, k.Z, k.R, GRAM_G1 | GRAM_D1 | GRAM_D2, gpart, sm.status);
      }
      Timed t(ex, KC_SMALL);
      lxl_zeta_beta(ex, L, gpart, np, sm);
    }
    // X += U alpha + zeta S, R -= zeta Z, P = R + (P - zeta V) beta
    {
      int np;
      {
        Timed t(ex, KC_AXPY);
        np = block_update_zeta<T>(ex, V, L, k.U, sm.alpha, k.S, k.Z, k.V, sm.zb, k.R, k.P, X64, npart);
      }
      Timed t(ex, KC_SMALL);
      lxl_norms(ex, L, npart, np, false, sm);
    }
    return check_launch(c, "iteration");
  }

  // The iteration as a CUDA graph: captured once per solve on the context's
  // stream (once the frozen step lengths are recorded, so that its launches no
  // longer change), then replayed with one launch.  Eager when profiling, when
  // MBICG_GRAPHS=0, or if capture fails.
  cudaGraphExec_t gexec = nullptr;
  long long graph_kernels = 0;
  bool graph_failed = false;
  int launch_iteration() {
    const char* env = getenv("MBICG_GRAPHS");
    const bool enabled = !(env && env[0] == '0');
    const bool stable = p.ncycle == 0 || p.domain_solver == MBICG_DOMAIN_SSOR || p.mr_mode != MBICG_MR_FROZEN ||
                        table_complete;
    if (!enabled || c->prof.on || !stable || graph_failed) return iteration_launches();
    if (!gexec) {
      const long long before = c->launches;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        const char* tr = getenv("MBICG_TRACE");
        if (tr && tr[0] == '1') fprintf(stderr, "mbicg: stream capture could not begin\n");
        cudaGetLastError();
        graph_failed = true;
        return iteration_launches();
      }
      const int rc = iteration_launches();
      cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (rc == MBICG_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      graph_kernels = c->launches - before;
      c->launches = before;
      if (rc != MBICG_OK || e != cudaSuccess || !gexec) {
        const char* tr = getenv("MBICG_TRACE");
        if (tr && tr[0] == '1')
          fprintf(stderr, "mbicg: iteration graph not used (status %d, %s; %s)\n", rc, cudaGetErrorString(e),
                  c->err.c_str());
        cudaGetLastError();
        c->err.clear();
        gexec = nullptr;
        graph_failed = true;
        return iteration_launches();
      }
    }
    CK(cudaGraphLaunch(gexec, c->stream));
    c->launches += graph_kernels;
    ++c->stats.graph_iterations;
    return MBICG_OK;
  }

  // The loop on the device: one captured CUDA graph whose WHILE conditional
  // node repeats the iteration and k_loop_control, which evaluates
  // Algorithm 2's WHILE test (and whether a reliable update is due) on the
  // device, so the host waits only when the loop stops.  Used where the
  // iteration graph is (and not with MBICG_DEVICE_LOOP=0); if it cannot be
  // built, the iteration graph with one host check per iteration is used.
  cudaGraphExec_t gloop = nullptr;
  cudaGraphConditionalHandle hcond = 0;
  long long loop_kernels = 0;  // kernels of one pass of the loop's body
  bool loop_failed = false;
  LoopCtl* dctl = nullptr;
  double* dbnorm = nullptr;
  double* dhist = nullptr;
  int hist_len = 0;
  std::vector<std::pair<int, int>> hist_ranges;  // iterations whose history is on the device

  bool loop_usable() const {
    const char* env = getenv("MBICG_GRAPHS");
    const char* dl = getenv("MBICG_DEVICE_LOOP");
    const bool stable = p.ncycle == 0 || p.domain_solver == MBICG_DOMAIN_SSOR || p.mr_mode != MBICG_MR_FROZEN ||
                        table_complete;
    return !(env && env[0] == '0') && !(dl && dl[0] == '0') && !c->prof.on && stable && !loop_failed &&
           !graph_failed;
  }

  int build_loop() {
    int rc;
    if ((rc = buf(c, "loop_ctl", 1, &dctl))) return rc;
    if ((rc = buf(c, "loop_bnorm", MAXL, &dbnorm))) return rc;
    hist_len = std::max(1, p.max_iter);
    if ((rc = buf(c, "loop_hist", (size_t)hist_len, &dhist))) return rc;
    memcpy(c->h_small + H_CTL_IN, bnorm, sizeof(double) * MAXL);
    CK(cudaMemcpyAsync(dbnorm, c->h_small + H_CTL_IN, sizeof(double) * MAXL, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));  // the pinned staging area is reused below
    cudaGraph_t g = nullptr;
    cudaGraphNode_t node = nullptr;
    cudaGraphNodeParams np = {};
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&hcond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hcond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    cudaGraph_t body = ok ? np.conditional.phGraph_out[0] : nullptr;
    const long long before = c->launches;
    if (ok)
      ok = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
    if (ok) {
      const int rc2 = iteration_launches();
      {
        Timed t(ex, KC_SMALL);
        loop_control(ex, dctl, sm.norms, dbnorm, sm.status, dhist, hist_len, hcond);
      }
      cudaGraph_t out = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->stream, &out);
      ok = rc2 == MBICG_OK && e == cudaSuccess && cudaGraphInstantiate(&gloop, g, 0) == cudaSuccess;
    }
    loop_kernels = c->launches - before;
    c->launches = before;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      const char* tr = getenv("MBICG_TRACE");
      if (tr && tr[0] == '1') fprintf(stderr, "mbicg: device loop not used (%s)\n", c->err.c_str());
      cudaGetLastError();
      c->err.clear();
      if (gloop) cudaGraphExecDestroy(gloop);
      gloop = nullptr;
      loop_failed = true;
    }
    return MBICG_OK;
  }

  // Iterations until the device's test stops the loop (at most max_iter - it);
  // returns the iterations done, the norms and status of the last one.
  int launch_loop(int it, double rmax_ru, int* done, int* st) {
    LoopCtl h{};
    h.it = it;
    h.max_iter = p.max_iter;
    h.Lc = std::min(L, Lc);
    h.sloppy = sizeof(T) == 4 ? 1 : 0;
    h.tol = tol_;
    h.delta_ru = p.delta_ru;
    h.rmax_ru = rmax_ru;
    h.relmax = 0;
    memcpy(c->h_small + H_CTL_IN, &h, sizeof(h));
    CK(cudaMemcpyAsync(dctl, c->h_small + H_CTL_IN, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    CK(cudaGraphLaunch(gloop, c->stream));
    CK(cudaMemcpyAsync(c->h_small + H_CTL_OUT, dctl, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    if (int rc = read_small(c, sm.norms, L, sm.status, h_norm, st)) return rc;
    memcpy(&h, c->h_small + H_CTL_OUT, sizeof(h));
    *done = h.it - it;
    if (*done < 1 || *done > p.max_iter) return fail(c, MBICG_ECUDA, "the device loop returned a bad iteration count");
    hist_ranges.push_back({it, *done});
    c->launches += (long long)*done * loop_kernels;
    c->stats.graph_iterations += *done;
    return MBICG_OK;
  }

  ~Solver() {
    if (gexec || gloop) cudaStreamSynchronize(c->stream);  // no replay of them still pending
    if (gexec) cudaGraphExecDestroy(gexec);
    if (gloop) cudaGraphExecDestroy(gloop);
  }

  double tol_ = 0;

  int run(const cx<double>* dB, cx<double>* dX, double tol, int* iters_out, double* true_res) {
    int rc;
    tol_ = tol;
    nl = (size_t)V * 12 * L;
    if ((rc = alloc())) return rc;
    // B, X into the internal layout
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<double>(ex, V, L, dB, B64);
      if (p.use_x0) abi_to_internal<double>(ex, V, L, dX, X64);
    }
    if (!p.use_x0) CK(cudaMemsetAsync(X64, 0, sizeof(cx<double>) * nl, c->stream));
    CK(cudaMemsetAsync(sm.status, 0, sizeof(int), c->stream));
    double rel[MAXL] = {0}, relmax;
    // R = B - A X
    if ((rc = true_residual(rel, &relmax, !p.use_x0))) return rc;
    // P = R, R~ = R
    CK(cudaMemcpyAsync(k.P, k.R, sizeof(cx<T>) * nl, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(k.Rt, k.R, sizeof(cx<T>) * nl, cudaMemcpyDeviceToDevice, c->stream));
    double rmax_ru = relmax;
    int it = 0, status = MBICG_OK;
    bool fresh_restart = false;
    int restarts_here = 0;  // restarts of this run (a continuation has its own)
    bool true_fresh = true;  // R holds B - A X from the FP64 operator
    const char* tr_env = getenv("MBICG_TRACE");
    const bool trace = tr_env && tr_env[0] == '1';
    const bool sloppy = sizeof(T) == 4;
    while (true) {
      if (!(relmax == relmax)) { status = MBICG_ENAN; break; }
      if (relmax <= tol) {
        // confirm on the true residual (FP32 loop: recompute; FP64: already exact to rounding)
        if (!sloppy || true_fresh) break;
        if ((rc = true_residual(rel, &relmax))) return rc;
        c->stats.reliable_updates++;
        rmax_ru = relmax;
        true_fresh = true;
        if (trace) fprintf(stderr, "mbicg: converged recursively, true max rel residual %.6e\n", relmax);
        if (relmax <= tol) break;
      }
      if (it >= p.max_iter) { status = MBICG_ENOTCONV; break; }
      int st = 0, ndone = 1;
      if (loop_usable() && !gloop) {
        if ((rc = build_loop())) return rc;
      }
      if (loop_usable() && gloop) {
        if ((rc = launch_loop(it, rmax_ru, &ndone, &st))) return rc;
      } else {
        if ((rc = launch_iteration())) return rc;
        if ((rc = read_small(c, sm.norms, L, sm.status, h_norm, &st))) return rc;
      }
      it += ndone;
      true_fresh = false;
      relmax = 0;
      for (int i = 0; i < L; ++i) {
        if (i == Lc) break;
        rel[i] = sqrt(h_norm[i]) / bnorm[i];
        if (!(rel[i] <= relmax)) relmax = rel[i];
      }
      if (p.res_history && it - 1 < p.res_history_len) p.res_history[it - 1] = relmax;
      if (trace) fprintf(stderr, "mbicg: iter %d (+%d) max rel residual %.6e status 0x%x\n", it, ndone, relmax, st);
      if (st & ST_TIMEOUT) return fail(c, MBICG_ECUDA, "a bounded wait for a bulk copy gave up in a kernel");
      if (st & ST_NAN) { status = MBICG_ENAN; break; }
      if (st) {
        // breakdown: restart from the current X (R = B - A X, P = R, R~ = R)
        if (fresh_restart || restarts_here >= 3) { status = MBICG_EBREAKDOWN; break; }
        ++restarts_here;
        c->stats.restarts++;
        CK(cudaMemsetAsync(sm.status, 0, sizeof(int), c->stream));
        if ((rc = true_residual(rel, &relmax))) return rc;
        CK(cudaMemcpyAsync(k.P, k.R, sizeof(cx<T>) * nl, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(k.Rt, k.R, sizeof(cx<T>) * nl, cudaMemcpyDeviceToDevice, c->stream));
        rmax_ru = relmax;
        fresh_restart = true;
        true_fresh = true;
        continue;
      }
      fresh_restart = false;
      // reliable update of the FP32 recursion
      if (sloppy && relmax > tol && relmax < p.delta_ru * rmax_ru) {
        if ((rc = true_residual(rel, &relmax))) return rc;
        if (trace) fprintf(stderr, "mbicg: reliable update, true max rel residual %.6e\n", relmax);
        c->stats.reliable_updates++;
        rmax_ru = relmax;
        true_fresh = true;
      }
    }
    // the recursive residuals of the iterations the device loop ran
    if (p.res_history && !hist_ranges.empty()) {
      CK(cudaStreamSynchronize(c->stream));
      for (const auto& r : hist_ranges) {
        const int n = std::min(r.first + r.second, p.res_history_len) - r.first;
        if (n > 0)
          CK(cudaMemcpy(p.res_history + r.first, dhist + r.first, sizeof(double) * n, cudaMemcpyDeviceToHost));
      }
    }
    // final true residual in FP64 (R is no longer needed)
    double trel[MAXL] = {0}, tmax;
    if (true_fresh || !sloppy) {
      if (!true_fresh) {
        if ((rc = true_residual(trel, &tmax))) return rc;
      } else {
        for (int i = 0; i < L; ++i) trel[i] = rel[i];
        tmax = relmax;
      }
    } else if ((rc = true_residual(trel, &tmax))) {
      return rc;
    }
    if (true_res)
      for (int i = 0; i < L; ++i) true_res[i] = trel[i];
    c->stats.true_res_max = tmax;
    c->stats.iters = it;
    if (iters_out) *iters_out = it;
    if (status == MBICG_OK && !(tmax <= tol)) status = MBICG_ENOTCONV;
    {
      Timed t(ex, KC_CONVERT);
      internal_to_abi<double>(ex, V, L, X64, dX);
    }
    if ((rc = check_launch(c, "solution"))) return rc;
    if (status == MBICG_ENOTCONV) fail(c, status, "not converged: max true residual %s", std::to_string(tmax).c_str());
    if (status == MBICG_EBREAKDOWN) fail(c, status, "breakdown (singular R~^H V, Tr(Z^H Z) = 0 or rank-deficient P)");
    if (status == MBICG_ENAN) fail(c, status, "NaN or Inf in a residual norm");
    return status;
  }
};

template <>
const cx<float>* Solver<float, float>::links_T() const { return c->U32; }
template <>
const cx<float>* Solver<float, float>::links_S() const { return c->U32; }
template <>
const cx<double>* Solver<double, float>::links_T() const { return c->U64; }
template <>
const cx<float>* Solver<double, float>::links_S() const { return c->U32; }
template <>
const cx<double>* Solver<double, double>::links_T() const { return c->U64; }
template <>
const cx<double>* Solver<double, double>::links_S() const { return c->U64; }
template <>
const cx<float>* Solver<float, double>::links_T() const { return c->U32; }
template <>
const cx<double>* Solver<float, double>::links_S() const { return c->U64; }

// solve: the block solve's parameters too; frozen: MBICG_MR_FROZEN allowed
// (the block solve, or a SAP call with a caller-held step-length table)
int check_params(mbicg_ctx* c, int L, const mbicg_params* p, bool solve, bool frozen) {
  if (L < 1 || L > MAXL) return fail(c, MBICG_EINVAL, "L must be in [1, 16]");
  if (!p) return fail(c, MBICG_EINVAL, "params is NULL");
  if (solve && (p->dummy_rhs < 0 || L + p->dummy_rhs > MAXL))
    return fail(c, MBICG_EINVAL, "dummy_rhs must be >= 0 with L + dummy_rhs <= 16");
  if (p->clover != 0 && p->clover != 1) return fail(c, MBICG_EINVAL, "clover must be 0 or 1");
  if (p->clover && !(c->csw > 0)) return fail(c, MBICG_EINVAL, "no clover term loaded");
  if (p->ncycle < 0 || p->ncycle > 64) return fail(c, MBICG_EINVAL, "ncycle out of range");
  if (p->ncycle > 0) {
    if (p->nmr < 1 || p->nmr > MAX_NMR) return fail(c, MBICG_EINVAL, "nmr must be in [1, 256]");
    if (!valid_blocking(c, p->block))
      return fail(c, MBICG_EINVAL, "SAP block must divide the lattice into an even number (>= 2) of domains per direction");
    if (p->domain_solver != MBICG_DOMAIN_MR && p->domain_solver != MBICG_DOMAIN_SSOR)
      return fail(c, MBICG_EINVAL, "bad domain_solver");
    if (p->domain_solver == MBICG_DOMAIN_SSOR) {
      if (p->nssor < 0 || p->nssor > 16) return fail(c, MBICG_EINVAL, "nssor must be in [0, 16]");
      if (!(p->ssor_omega > 0 && p->ssor_omega < 2)) return fail(c, MBICG_EINVAL, "ssor_omega must be in (0, 2)");
    } else if (p->mr_mode < 0 || p->mr_mode > 2 || (!frozen && p->mr_mode == MBICG_MR_FROZEN)) {
      return fail(c, MBICG_EINVAL, "bad mr_mode");
    }
    if (p->prec_sap != MBICG_FP32 && p->prec_sap != MBICG_FP64 && p->prec_sap != MBICG_FP16)
      return fail(c, MBICG_EINVAL, "prec_sap must be MBICG_FP32, MBICG_FP64 or MBICG_FP16");
    if (p->prec_sap == MBICG_FP16) {
      if (p->domain_solver != MBICG_DOMAIN_MR || p->mr_mode == MBICG_MR_BLOCK || p->clover)
        return fail(c, MBICG_EINVAL, "FP16 storage of the preconditioner takes MR domain solves with "
                                     "MBICG_MR_COLUMN or MBICG_MR_FROZEN and the Wilson matrix");
      Geom g16 = lattice_geom(c, p->block);
      g16.su3 = 1;
      if (!sap_sweep_fusable(g16, 3) || (c->gauge && !c->su3))
        return fail(c, MBICG_EINVAL, "FP16 storage of the preconditioner needs 8^4 or 4^4 domains and SU(3) links");
    }
  }
  if (solve) {
    if (p->prec_D != MBICG_FP32 && p->prec_D != MBICG_FP64)
      return fail(c, MBICG_EINVAL, "prec_D must be MBICG_FP32 or MBICG_FP64");
    if (p->ncycle > 0 && p->prec_sap == MBICG_FP16 && p->prec_D != MBICG_FP32)
      return fail(c, MBICG_EINVAL, "FP16 storage of the preconditioner needs prec_D = MBICG_FP32");
    if (p->max_iter < 0) return fail(c, MBICG_EINVAL, "max_iter < 0");
    if (!(p->delta_ru > 0 && p->delta_ru < 1)) return fail(c, MBICG_EINVAL, "delta_ru must be in (0, 1)");
  }
  return MBICG_OK;
}

template <typename T, typename TS>
int run_solve(mbicg_ctx* c, const cx<double>* dB, cx<double>* dX, int L, double kappa, double tol,
              const mbicg_params* p, const double* bnorm, int* iters, double* true_res, bool keep_table = false,
              int Lc = 0) {
  Solver<T, TS> s;
  s.keep_table = keep_table;
  s.Lc = Lc > 0 ? Lc : L;
  s.c = c;
  s.ex = exec_of(c);
  s.g = lattice_geom(c, p->ncycle > 0 ? p->block : nullptr);
  s.L = L;
  s.kappa = kappa;
  s.p = *p;
  s.V = c->V;
  if (p->clover) {
    s.ti64 = c->Ti64;
    s.ti32 = c->Ti32;
  }
  s.sap16 = p->ncycle > 0 && p->prec_sap == MBICG_FP16 && std::is_same<T, float>::value;
  for (int i = 0; i < L; ++i) s.bnorm[i] = bnorm[i];
  return s.run(dB, dX, tol, iters, true_res);
}

// T^{-1} = (1 + kappa C)^{-1} of the loaded clover term, formed when kappa changes
int clover_for_kappa(mbicg_ctx* c, double kappa) {
  if (!(c->csw > 0)) return fail(c, MBICG_EINVAL, "no clover term loaded");
  if (c->tinv_kappa == kappa) return MBICG_OK;
  int* st;
  int rc;
  if ((rc = buf(c, "clover_status", 1, &st))) return rc;
  CK(cudaMemsetAsync(st, 0, sizeof(int), c->stream));
  const Exec ex = exec_of(c);
  {
    Timed t(ex, KC_CONVERT);
    clover_terms(ex, c->V, c->C64, kappa, c->Ti64, c->Ti32, c->C32, st);
  }
  if ((rc = check_launch(c, "clover_terms"))) return rc;
  CK(cudaMemcpyAsync(c->h_small, st, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int bad = 0;
  memcpy(&bad, c->h_small, sizeof(int));
  if (bad) {
    c->tinv_kappa = NAN;
    return fail(c, MBICG_EINVAL, "1 + kappa C is singular at some site");
  }
  c->tinv_kappa = kappa;
  return MBICG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
cudaStream_t mbicg::ctx_stream(const mbicg_ctx* c) { return c->stream; }

size_t mbicg::ctx_workspace_bytes(const mbicg_ctx* c) {
  size_t n = 0;
  for (const auto& kv : c->bufs) n += kv.second.second < 256 ? 256 : kv.second.second;
  return n;
}

void mbicg::ctx_release_workspace(mbicg_ctx* c) {
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->bufs) cudaFree(kv.second.first);
  c->bufs.clear();
}

extern "C" {

void mbicg_default_params(mbicg_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->ncycle = 4;
  p->nmr = 4;
  for (int mu = 0; mu < 4; ++mu) p->block[mu] = 4;
  p->mr_mode = MBICG_MR_FROZEN;
  p->prec_sap = MBICG_FP32;
  p->prec_D = MBICG_FP32;
  p->max_iter = 1000;
  p->use_x0 = 0;
  p->delta_ru = 0.1;
  p->res_history = nullptr;
  p->res_history_len = 0;
  p->domain_solver = MBICG_DOMAIN_MR;
  p->nssor = 1;
  p->ssor_omega = 1.26;
}

int mbicg_create(mbicg_ctx** out, const int dims[4], int device, void* cuda_stream) {
  if (!out) return MBICG_EINVAL;
  *out = nullptr;
  if (!dims) return MBICG_EINVAL;
  long long vol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 2 || dims[mu] % 2 != 0 || dims[mu] > 4096) return MBICG_EINVAL;
    vol *= dims[mu];
  }
  if (vol > (1ll << 27)) return MBICG_EINVAL;  // 32-bit site and (site, rhs) indices
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MBICG_ECUDA;
  }
  mbicg_ctx* c = new mbicg_ctx();
  c->device = device;
  c->V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    c->dims[mu] = dims[mu];
    c->V *= dims[mu];
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return MBICG_ECUDA;
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return MBICG_ECUDA;
    }
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->h_small, sizeof(double) * H_SMALL) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return MBICG_ENOMEM;
  }
  *out = c;
  return MBICG_OK;
}

void mbicg_destroy(mbicg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->bufs) cudaFree(kv.second.first);
  if (c->U64) cudaFree(c->U64);
  if (c->U32) cudaFree(c->U32);
  if (c->U16) cudaFree(c->U16);
  if (c->U12) cudaFree(c->U12);
  if (c->C64) cudaFree(c->C64);
  if (c->C32) cudaFree(c->C32);
  if (c->Ti64) cudaFree(c->Ti64);
  if (c->Ti32) cudaFree(c->Ti32);
  c->prof.release();
  if (c->h_small) cudaFreeHost(c->h_small);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

int mbicg_load_gauge(mbicg_ctx* c, const double* U) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  if (!U) return fail(c, MBICG_EINVAL, "U is NULL");
  CK(cudaSetDevice(c->device));
  // the copies are overwritten below: until they all hold the new field, no
  // field is loaded
  c->gauge = false;
  c->su3 = false;
  c->launches = 0;
  c->csw = 0.0;  // a clover term belongs to the previous field
  c->tinv_kappa = NAN;
  const size_t n = (size_t)c->V * 36;  // complex numbers
  if (!c->U64) CK(cudaMalloc(&c->U64, sizeof(cx<double>) * n));
  if (!c->U32) CK(cudaMalloc(&c->U32, sizeof(cx<float>) * n));
  if (!c->U16) CK(cudaMalloc(&c->U16, sizeof(__half2) * (size_t)c->V * 24));
  if (!c->U12) CK(cudaMalloc(&c->U12, sizeof(cx<float>) * (size_t)c->V * 24));
  Staged s;
  int rc = stage_in(c, U, sizeof(cx<double>) * n, "gauge_stage", true, &s);
  if (rc) return rc;
  int* flag;
  if ((rc = buf(c, "gauge_flag", 1, &flag))) return rc;
  CK(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  const Exec ex = exec_of(c);
  {
    Timed t(ex, KC_CONVERT);
    convert_links(ex, c->V, static_cast<const cx<double>*>(s.dev), c->U64, c->U32, flag);
    links_to_half(ex, c->V, static_cast<const cx<double>*>(s.dev), c->U16);
    links_to_rows(ex, c->V, c->U32, c->U12);
  }
  if ((rc = check_launch(c, "load_gauge"))) return rc;
  int bad = 0;
  CK(cudaMemcpyAsync(c->h_small, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->prof.collect();
  memcpy(&bad, c->h_small, sizeof(int));
  c->stats.kernel_launches = c->launches;
  if (bad & 1) return fail(c, MBICG_ENAN, "gauge field holds NaN or Inf");
  c->su3 = (bad & 2) == 0;
  c->gauge = true;
  return MBICG_OK;
}

int mbicg_apply_D(mbicg_ctx* c, const double* in, double* out, int L, double kappa, int prec) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  if (!in || !out || in == out) return fail(c, MBICG_EINVAL, "in/out NULL or aliased");
  if (L < 1 || L > MAXL) return fail(c, MBICG_EINVAL, "L must be in [1, 16]");
  if (prec != MBICG_FP64 && prec != MBICG_FP32 && prec != MBICG_FP16)
    return fail(c, MBICG_EINVAL, "prec must be FP64, FP32 or FP16");
  if (!c->gauge) return fail(c, MBICG_ENOGAUGE, "no gauge field loaded");
  if (prec == MBICG_FP16 && !c->su3)
    return fail(c, MBICG_EINVAL, "FP16 storage keeps two link rows and needs SU(3) links");
  CK(cudaSetDevice(c->device));
  c->launches = 0;
  const size_t nl = (size_t)c->V * 12 * L;
  Staged si, so;
  int rc;
  if ((rc = stage_in(c, in, sizeof(cx<double>) * nl, "abi_in", true, &si))) return rc;
  if ((rc = stage_in(c, out, sizeof(cx<double>) * nl, "abi_out", false, &so))) return rc;
  const Exec ex = exec_of(c);
  const Geom g = lattice_geom(c, nullptr);
  if (prec == MBICG_FP64) {
    cx<double>*a, *b;
    if ((rc = buf(c, "op64_a", nl, &a)) || (rc = buf(c, "op64_b", nl, &b))) return rc;
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<double>(ex, c->V, L, static_cast<const cx<double>*>(si.dev), a);
    }
    {
      Timed t(ex, KC_DSLASH64);
      dslash_full<double>(ex, g, c->U64, a, b, L, kappa);
    }
    Timed t(ex, KC_CONVERT);
    internal_to_abi<double>(ex, c->V, L, b, static_cast<cx<double>*>(so.dev));
  } else if (prec == MBICG_FP16) {
    // FP16 blocks (48 bytes per spinor) and their scales, carved from FP32-sized buffers
    cx<float>*a, *b;
    float *sa, *sb;
    if ((rc = buf(c, "op16_a", nl / 2, &a)) || (rc = buf(c, "op16_b", nl / 2, &b))) return rc;
    if ((rc = buf(c, "op16_sa", (size_t)c->V * L, &sa)) || (rc = buf(c, "op16_sb", (size_t)c->V * L, &sb))) return rc;
    __half2* qa = reinterpret_cast<__half2*>(a);
    __half2* qb = reinterpret_cast<__half2*>(b);
    {
      Timed t(ex, KC_CONVERT);
      abi_to_half(ex, c->V, L, static_cast<const cx<double>*>(si.dev), qa, sa);
    }
    {
      Timed t(ex, KC_DSLASH);
      dslash_half(ex, g, c->U16, qa, sa, qb, sb, L, kappa);
    }
    Timed t(ex, KC_CONVERT);
    half_to_abi(ex, c->V, L, qb, sb, static_cast<cx<double>*>(so.dev));
  } else {
    cx<float>*a, *b;
    if ((rc = buf(c, "op32_a", nl, &a)) || (rc = buf(c, "op32_b", nl, &b))) return rc;
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<float>(ex, c->V, L, static_cast<const cx<double>*>(si.dev), a);
    }
    {
      Timed t(ex, KC_DSLASH);
      dslash_full<float>(ex, g, c->U32, a, b, L, kappa, nullptr, 0, links12(c));
    }
    Timed t(ex, KC_CONVERT);
    internal_to_abi<float>(ex, c->V, L, b, static_cast<cx<double>*>(so.dev));
  }
  if ((rc = check_launch(c, "apply_D"))) return rc;
  if ((rc = stage_out(c, so))) return rc;
  c->stats.kernel_launches = c->launches;
  return MBICG_OK;
}

int mbicg_load_clover(mbicg_ctx* c, double csw) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  if (!(csw >= 0) || !isfinite(csw)) return fail(c, MBICG_EINVAL, "csw must be finite and >= 0");
  if (!c->gauge) return fail(c, MBICG_ENOGAUGE, "no gauge field loaded");
  CK(cudaSetDevice(c->device));
  c->launches = 0;
  c->tinv_kappa = NAN;
  c->csw = 0.0;
  if (csw == 0) return MBICG_OK;
  const size_t n = (size_t)c->V * HERM_PER_SITE;
  if (!c->C64) CK(cudaMalloc(&c->C64, sizeof(double) * n));
  if (!c->C32) CK(cudaMalloc(&c->C32, sizeof(float) * n));
  if (!c->Ti64) CK(cudaMalloc(&c->Ti64, sizeof(double) * n));
  if (!c->Ti32) CK(cudaMalloc(&c->Ti32, sizeof(float) * n));
  const Exec ex = exec_of(c);
  {
    Timed t(ex, KC_CONVERT);
    clover_field(ex, lattice_geom(c, nullptr), c->U64, csw, c->C64);
  }
  int rc;
  if ((rc = check_launch(c, "load_clover"))) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->prof.collect();
  c->csw = csw;
  c->stats.kernel_launches = c->launches;
  return MBICG_OK;
}

int mbicg_apply_clover(mbicg_ctx* c, const double* in, double* out, int L, double kappa, int prec, int jacobi) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  if (!in || !out || in == out) return fail(c, MBICG_EINVAL, "in/out NULL or aliased");
  if (L < 1 || L > MAXL) return fail(c, MBICG_EINVAL, "L must be in [1, 16]");
  if (prec != MBICG_FP64 && prec != MBICG_FP32) return fail(c, MBICG_EINVAL, "prec must be FP64 or FP32");
  if (jacobi != 0 && jacobi != 1) return fail(c, MBICG_EINVAL, "jacobi must be 0 or 1");
  if (!c->gauge) return fail(c, MBICG_ENOGAUGE, "no gauge field loaded");
  CK(cudaSetDevice(c->device));
  c->launches = 0;
  int rc;
  if ((rc = clover_for_kappa(c, kappa))) return rc;
  const size_t nl = (size_t)c->V * 12 * L;
  Staged si, so;
  if ((rc = stage_in(c, in, sizeof(cx<double>) * nl, "abi_in", true, &si))) return rc;
  if ((rc = stage_in(c, out, sizeof(cx<double>) * nl, "abi_out", false, &so))) return rc;
  const Exec ex = exec_of(c);
  const Geom g = lattice_geom(c, nullptr);
  const int cm = jacobi ? 1 : 2;
  if (prec == MBICG_FP64) {
    cx<double>*a, *b;
    if ((rc = buf(c, "op64_a", nl, &a)) || (rc = buf(c, "op64_b", nl, &b))) return rc;
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<double>(ex, c->V, L, static_cast<const cx<double>*>(si.dev), a);
    }
    {
      Timed t(ex, KC_DSLASH64);
      dslash_full<double>(ex, g, c->U64, a, b, L, kappa, jacobi ? c->Ti64 : c->C64, cm);
    }
    Timed t(ex, KC_CONVERT);
    internal_to_abi<double>(ex, c->V, L, b, static_cast<cx<double>*>(so.dev));
  } else {
    cx<float>*a, *b;
    if ((rc = buf(c, "op32_a", nl, &a)) || (rc = buf(c, "op32_b", nl, &b))) return rc;
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<float>(ex, c->V, L, static_cast<const cx<double>*>(si.dev), a);
    }
    {
      Timed t(ex, KC_DSLASH);
      dslash_full<float>(ex, g, c->U32, a, b, L, kappa, jacobi ? c->Ti32 : c->C32, cm);
    }
    Timed t(ex, KC_CONVERT);
    internal_to_abi<float>(ex, c->V, L, b, static_cast<cx<double>*>(so.dev));
  }
  if ((rc = check_launch(c, "apply_clover"))) return rc;
  if ((rc = stage_out(c, so))) return rc;
  c->stats.kernel_launches = c->launches;
  return MBICG_OK;
}

}  // extern "C"

namespace {

// Lexicographic index of the k-th domain of colour `colour` (the enumeration
// of colour_domain in common.cuh).
long long colour_domain_lex(const Geom& g, int colour, int k) {
  const int half = g.nb[0] / 2;
  const int row0 = k / half;
  const int j = 2 * (k - row0 * half);
  int b[4];
  b[1] = row0 % g.nb[1];
  const int row1 = row0 / g.nb[1];
  b[2] = row1 % g.nb[2];
  b[3] = row1 / g.nb[2];
  b[0] = j + (colour ^ ((b[1] + b[2] + b[3]) & 1));
  return b[0] + (long long)g.nb[0] * (b[1] + (long long)g.nb[1] * (b[2] + (long long)g.nb[2] * b[3]));
}

// out = M_SAP in.  table_lex != NULL: frozen MR step lengths held by the
// caller (host, complex [ncycle][2][nmr][nd], lexicographic domain index):
// entries still NaN are recorded by this call and written back, and once
// every entry the sweeps use is set the table is replayed (the solver's path).
int sap_precond_impl(mbicg_ctx* c, const double* in, double* out, int L, double kappa, const mbicg_params* p,
                     double* table_lex, int* complete) {
  if (!in || !out || in == out) return fail(c, MBICG_EINVAL, "in/out NULL or aliased");
  int rc;
  if ((rc = check_params(c, L, p, false, table_lex != nullptr))) return rc;
  if (p->ncycle < 1) return fail(c, MBICG_EINVAL, "ncycle must be >= 1");
  if (table_lex && (p->domain_solver != MBICG_DOMAIN_MR || p->mr_mode != MBICG_MR_FROZEN))
    return fail(c, MBICG_EINVAL, "a step-length table needs MR domain solves with mr_mode MBICG_MR_FROZEN");
  if (!c->gauge) return fail(c, MBICG_ENOGAUGE, "no gauge field loaded");
  CK(cudaSetDevice(c->device));
  c->launches = 0;
  if (p->clover && (rc = clover_for_kappa(c, kappa))) return rc;
  const size_t nl = (size_t)c->V * 12 * L;
  Staged si, so;
  if ((rc = stage_in(c, in, sizeof(cx<double>) * nl, "abi_in", true, &si))) return rc;
  if ((rc = stage_in(c, out, sizeof(cx<double>) * nl, "abi_out", false, &so))) return rc;
  const Exec ex = exec_of(c);
  const Geom g = lattice_geom(c, p->block);
  const int ndc = g.nd / 2;
  // the caller's table in the library's layout, complex [ncycle][2][nmr][nd / 2]
  const size_t ntab = (size_t)p->ncycle * 2 * p->nmr * ndc;
  std::vector<double> htab;
  double* dtab = nullptr;
  int* unset = nullptr;
  int mode = p->mr_mode;
  if (table_lex) {
    htab.resize(2 * ntab);
    bool any_nan = false;
    for (int cyc = 0; cyc < p->ncycle; ++cyc)
      for (int col = 0; col < 2; ++col)
        for (int it = 0; it < p->nmr; ++it)
          for (int k = 0; k < ndc; ++k) {
            const size_t row = ((size_t)cyc * 2 + col) * p->nmr + it;
            const size_t src = (row * g.nd + colour_domain_lex(g, col, k)) * 2;
            const size_t dst = (row * ndc + k) * 2;
            htab[dst] = table_lex[src];
            htab[dst + 1] = table_lex[src + 1];
            any_nan = any_nan || isnan(htab[dst]) || isnan(htab[dst + 1]);
          }
    if ((rc = buf(c, "sapp_table", 2 * ntab, &dtab))) return rc;
    if ((rc = buf(c, "sapp_unset", 1, &unset))) return rc;
    CK(cudaMemcpyAsync(dtab, htab.data(), sizeof(double) * 2 * ntab, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(unset, 0, sizeof(int), c->stream));
    mode = any_nan ? 2 : 3;  // record where unset, else replay
  }
  auto run = [&](auto tag, const auto* links) -> int {
    using R = decltype(tag);
    cx<R>*a, *b, *r, *q, *x;
    SapWork w;
    int rc2;
    if ((rc2 = buf(c, "sapp_a", nl, &a))) return rc2;
    if ((rc2 = buf(c, "sapp_b", nl, &b))) return rc2;
    if ((rc2 = buf(c, "sap_r", nl, &r))) return rc2;
    if ((rc2 = buf(c, "sap_q", nl, &q))) return rc2;
    if ((rc2 = buf(c, "sap_x", nl, &x))) return rc2;
    w.r = r;
    w.q = q;
    w.x = x;
    const int S = sap_sites_per_cta(g, L, sizeof(R) == 8);
    if ((rc2 = buf(c, "sap_dots", (size_t)ndc * (g.Vd / S) * L * 3, &w.dots))) return rc2;
    if ((rc2 = buf(c, "sap_omega", (size_t)ndc * L * 2, &w.omega))) return rc2;
    const SsorParams sp{p->nssor, p->ssor_omega};
    if (p->domain_solver == MBICG_DOMAIN_SSOR) {
      const char* names4[4] = {"ssor_acc", "ssor_term", "ssor_pv", "ssor_pqv"};
      for (int i = 0; i < 4; ++i) {
        cx<R>* b4;
        if ((rc2 = buf(c, names4[i], nl, &b4))) return rc2;
        w.ssor[i] = b4;
      }
      if ((rc2 = buf(c, "ssor_levels", (size_t)g.Vd, &w.levels))) return rc2;
      if (sap_prepare_ssor(g, w, c->stream) != cudaSuccess) return fail(c, MBICG_ECUDA, "ssor level table");
    }
    {
      Timed t(ex, KC_CONVERT);
      abi_to_internal<R>(ex, c->V, L, static_cast<const cx<double>*>(si.dev), a);
    }
    const R* tinv = nullptr;
    if (p->clover) tinv = reinterpret_cast<const R*>(sizeof(R) == 8 ? static_cast<const void*>(c->Ti64)
                                                                     : static_cast<const void*>(c->Ti32));
    bool done = false;
    if constexpr (std::is_same<R, float>::value) {
      if (p->prec_sap == MBICG_FP16 && (mode == 0 || mode == 3)) {
        // FP16 storage of the preconditioner's blocks (a table still being
        // recorded is recorded by the FP32 path below)
        SapHalf h{};
        const size_t nsp = (size_t)c->V * L;
        if ((rc2 = buf(c, "h16_eta", nl, &h.eta)) || (rc2 = buf(c, "h16_eta_sc", nsp, &h.eta_sc)) ||
            (rc2 = buf(c, "h16_psi", nl, &h.psi)) || (rc2 = buf(c, "h16_psi_sc", nsp, &h.psi_sc)) ||
            (rc2 = buf(c, "h16_r", nl, &h.r)) || (rc2 = buf(c, "h16_r_sc", nsp, &h.r_sc)))
          return rc2;
        {
          Timed t(ex, KC_CONVERT);
          block_to_half(ex, (long long)nsp, a, h.eta, h.eta_sc);
        }
        sap_apply_h(ex, g, links, h, L, kappa, p->ncycle, p->nmr, mode, dtab);
        Timed t(ex, KC_CONVERT);
        half_to_block(ex, (long long)nsp, h.psi, h.psi_sc, b);
        done = true;
      }
    }
    if (std::is_same<R, float>::value) w.links12 = links12(c);
    if (!done)
      sap_apply<R>(ex, g, links, a, b, L, kappa, p->ncycle, p->nmr, mode, dtab, unset, w, tinv,
                   p->domain_solver == MBICG_DOMAIN_SSOR ? &sp : nullptr);
    Timed t(ex, KC_CONVERT);
    internal_to_abi<R>(ex, c->V, L, b, static_cast<cx<double>*>(so.dev));
    // the level table's host copy lives in w: wait for its upload before w goes
    if (p->domain_solver == MBICG_DOMAIN_SSOR && cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(c, MBICG_ECUDA, "sap_precond");
    return MBICG_OK;
  };
  if (p->prec_sap == MBICG_FP64) rc = run(double(0), c->U64);
  else rc = run(float(0), c->U32);
  if (rc) return rc;
  if ((rc = check_launch(c, "sap_precond"))) return rc;
  if ((rc = stage_out(c, so))) return rc;
  if (table_lex) {
    // the recorded entries back into the caller's table
    CK(cudaMemcpyAsync(htab.data(), dtab, sizeof(double) * 2 * ntab, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    bool all_set = true;
    for (int cyc = 0; cyc < p->ncycle; ++cyc)
      for (int col = 0; col < 2; ++col)
        for (int it = 0; it < p->nmr; ++it)
          for (int k = 0; k < ndc; ++k) {
            const size_t row = ((size_t)cyc * 2 + col) * p->nmr + it;
            const size_t dst = (row * g.nd + colour_domain_lex(g, col, k)) * 2;
            const size_t src = (row * ndc + k) * 2;
            table_lex[dst] = htab[src];
            table_lex[dst + 1] = htab[src + 1];
            all_set = all_set && !isnan(htab[src]);
          }
    if (complete) *complete = all_set ? 1 : 0;
  }
  c->stats.kernel_launches = c->launches;
  return MBICG_OK;
}

}  // namespace

extern "C" {

int mbicg_sap_precond(mbicg_ctx* c, const double* in, double* out, int L, double kappa, const mbicg_params* p) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  return sap_precond_impl(c, in, out, L, kappa, p, nullptr, nullptr);
}

int mbicg_sap_table_len(const mbicg_ctx* c, const mbicg_params* p, long long* n_doubles) {
  if (!c || !p || !n_doubles) return MBICG_EINVAL;
  mbicg_ctx* m = const_cast<mbicg_ctx*>(c);
  m->err.clear();
  if (p->ncycle < 1 || p->nmr < 1) return fail(m, MBICG_EINVAL, "ncycle and nmr must be >= 1");
  if (!valid_blocking(c, p->block))
    return fail(m, MBICG_EINVAL, "SAP block must divide the lattice into an even number (>= 2) of domains per direction");
  long long nd = 1;
  for (int mu = 0; mu < 4; ++mu) nd *= c->dims[mu] / p->block[mu];
  *n_doubles = 2LL * p->ncycle * 2 * p->nmr * nd;
  return MBICG_OK;
}

int mbicg_sap_precond_frozen(mbicg_ctx* c, const double* in, double* out, int L, double kappa,
                             const mbicg_params* p, double* table, int* complete) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  if (!table) return fail(c, MBICG_EINVAL, "table is NULL");
  if (is_device_ptr(table)) return fail(c, MBICG_EINVAL, "table must be host memory");
  return sap_precond_impl(c, in, out, L, kappa, p, table, complete);
}

int mbicg_block_solve(mbicg_ctx* c, const double* B, double* X, int L, double kappa, double tol,
                      const mbicg_params* p, int* iters, double* true_res) {
  if (!c) return MBICG_EINVAL;
  c->err.clear();
  c->stats = mbicg_stats{};
  if (!B || !X || (const void*)B == (const void*)X) return fail(c, MBICG_EINVAL, "B/X NULL or aliased");
  int rc;
  if ((rc = check_params(c, L, p, true, true))) return rc;
  if (!(tol > 0)) return fail(c, MBICG_EINVAL, "tol must be > 0");
  if (!c->gauge) return fail(c, MBICG_ENOGAUGE, "no gauge field loaded");
  CK(cudaSetDevice(c->device));
  c->launches = 0;
  const size_t nl = (size_t)c->V * 12 * L;
  Staged sb, sx;
  if ((rc = stage_in(c, B, sizeof(cx<double>) * nl, "abi_in", true, &sb))) return rc;
  if ((rc = stage_in(c, X, sizeof(cx<double>) * nl, "abi_out", p->use_x0 != 0, &sx))) return rc;
  double bnorm[MAXL];
  bool bad = false;
  if ((rc = abi_norms(c, static_cast<const cx<double>*>(sb.dev), L, bnorm, &bad))) return rc;
  if (bad) return fail(c, MBICG_ENAN, "B holds NaN or Inf");
  for (int i = 0; i < L; ++i)
    if (!(bnorm[i] > 0)) return fail(c, MBICG_EINVAL, "B has a zero column");
  if (p->use_x0) {
    double xn[MAXL];
    if ((rc = abi_norms(c, static_cast<const cx<double>*>(sx.dev), L, xn, &bad))) return rc;
    if (bad) return fail(c, MBICG_ENAN, "X0 holds NaN or Inf");
  }
  const cx<double>* dB = static_cast<const cx<double>*>(sb.dev);
  cx<double>* dX = static_cast<cx<double>*>(sx.dev);
  if (p->clover) {
    // D_c X = B is solved as A X = T^{-1} B with A = T^{-1} D_c
    if ((rc = clover_for_kappa(c, kappa))) return rc;
    cx<double>* Bc;
    if ((rc = buf(c, "clover_B", nl, &Bc))) return rc;
    clover_abi(exec_of(c), c->V, L, c->Ti64, dB, Bc);
    if ((rc = abi_norms(c, Bc, L, bnorm, &bad))) return rc;
    for (int i = 0; i < L; ++i)
      if (!(bnorm[i] > 0)) return fail(c, MBICG_EINVAL, "T^{-1} B has a zero column");
    dB = Bc;
  }
  // dummy right-hand sides: solve the block widened by seeded Gaussian
  // columns; the stopping test and the results cover the first L columns
  const int Lt = L + p->dummy_rhs;
  double tres_all[MAXL] = {0};
  if (p->dummy_rhs > 0) {
    const Exec ex = exec_of(c);
    const size_t nlt = (size_t)c->V * 12 * Lt;
    cx<double>*Bt, *Xt;
    if ((rc = buf(c, "dummy_B", nlt, &Bt)) || (rc = buf(c, "dummy_X", nlt, &Xt))) return rc;
    {
      Timed t(ex, KC_CONVERT);
      pack_dummies(ex, c->V, L, Lt, dB, Bt, p->dummy_seed, true);
    }
    if (p->use_x0) {
      Timed t(ex, KC_CONVERT);
      pack_dummies(ex, c->V, L, Lt, dX, Xt, 0, false);
    }
    if ((rc = abi_norms(c, Bt, Lt, bnorm, &bad))) return rc;
    dB = Bt;
    dX = Xt;
  }
  const bool sap64 = p->ncycle > 0 && p->prec_sap == MBICG_FP64;
  int st;
  if (p->prec_D == MBICG_FP64) {
    st = sap64 ? run_solve<double, double>(c, dB, dX, Lt, kappa, tol, p, bnorm, iters, tres_all, false, L)
               : run_solve<double, float>(c, dB, dX, Lt, kappa, tol, p, bnorm, iters, tres_all, false, L);
  } else {
    st = sap64 ? run_solve<float, double>(c, dB, dX, Lt, kappa, tol, p, bnorm, iters, tres_all, false, L)
               : run_solve<float, float>(c, dB, dX, Lt, kappa, tol, p, bnorm, iters, tres_all, false, L);
    if (st == MBICG_EBREAKDOWN) {
      // The FP32 Krylov vectors lost the rank of the search block again after
      // every restart: continue from the current X with FP64 Krylov vectors
      // (the FP32 preconditioner with its frozen step lengths stays), for the
      // iterations that remain.
      const mbicg_stats first = c->stats;
      mbicg_params q = *p;
      q.use_x0 = 1;
      q.max_iter = std::max(1, p->max_iter - first.iters);
      c->err.clear();
      int it2 = 0;
      // the same preconditioner: the frozen MR step lengths recorded so far are kept
      st = sap64 ? run_solve<double, double>(c, dB, dX, Lt, kappa, tol, &q, bnorm, &it2, tres_all, true, L)
                 : run_solve<double, float>(c, dB, dX, Lt, kappa, tol, &q, bnorm, &it2, tres_all, true, L);
      c->stats.iters = first.iters + it2;
      c->stats.precision_fallbacks = 1;
      if (iters) *iters = first.iters + it2;
    }
  }
  if (true_res)
    for (int i = 0; i < L; ++i) true_res[i] = tres_all[i];
  if (p->dummy_rhs > 0 && (st == MBICG_OK || st == MBICG_ENOTCONV || st == MBICG_EBREAKDOWN)) {
    const Exec ex = exec_of(c);
    Timed t(ex, KC_CONVERT);
    first_columns(ex, c->V, Lt, L, dX, static_cast<cx<double>*>(sx.dev));
  }
  if (st == MBICG_ECUDA || st == MBICG_ENOMEM || st == MBICG_EINVAL) return st;
  if ((rc = stage_out(c, sx))) return rc;
  if (!sx.host) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "block_solve");
  }
  c->prof.collect();
  c->stats.kernel_launches = c->launches;
  return st;
}

int mbicg_get_stats(const mbicg_ctx* c, mbicg_stats* out) {
  if (!c || !out) return MBICG_EINVAL;
  *out = c->stats;
  return MBICG_OK;
}

int mbicg_set_profiling(mbicg_ctx* c, int enable) {
  if (!c) return MBICG_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->prof.collect();
  c->prof.reset();
  c->prof.on = enable != 0;
  return MBICG_OK;
}

int mbicg_get_profile(const mbicg_ctx* c, double* ms, long long* launches, int n) {
  if (!c || n < 0 || n > MBICG_K_NCLASS) return MBICG_EINVAL;
  mbicg_ctx* m = const_cast<mbicg_ctx*>(c);
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  m->prof.collect();
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = c->prof.ms[i];
    if (launches) launches[i] = c->prof.count[i];
  }
  return MBICG_OK;
}

const char* mbicg_last_error(const mbicg_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
