// Threaded host emulation of the library's block linear algebra kernels: the
// Gram kernel (bulk copies into shared memory, mbarrier waits), the row
// kernels of the block updates and the one-CTA L x L kernels, each run with
// the launch shape the library uses.  blas_parts.inc is cut out of the CUDA
// sources by the test.
#include "blas_parts.inc"

thread_local EmuThread emu_t;
EmuDim blockDim, gridDim;
int emu_bad_access = 0;

using namespace mbicg;
using namespace mbicg::emu_blas;

template <typename F>
static void one_cta(int threads, F k) { emu_launch(1, 1, threads, 0, k); }

template <typename R, int L>
static int gram(long long nsite, const void* A, const void* B1, const void* B2, int flags, double* part) {
  long long launches = 0;
  const Exec ex{nullptr, &launches, nullptr};
  int err = 0;
  emu_mbar_reset();
  const int n = launch_gram<R, L>(ex, nsite, (const cx<R>*)A, (const cx<R>*)B1, (const cx<R>*)B2, flags, part, &err);
  return err ? -err : n;
}

template <typename R, int L>
static void updates(int which, int ncta, int nrow, const void* U, const double* alpha, const void* S, const void* Z,
                    const void* V, const double* zb, void* Rv, void* P, void* X, double* part, const double* M,
                    void* Y) {
  using C = cx<R>;
  if (which == 0)
    emu_launch(ncta, 1, NT, 0, [&] { k_transform<R, L>(nrow, (const C*)U, M, (C*)Y); });
  else if (which == 1)
    emu_launch(ncta, 1, NT, 0, [&] { k_update_alpha<R, L>(nrow, (const C*)V, alpha, (C*)Rv); });
  else
    emu_launch(ncta, 1, NT, 0, [&] {
      k_update_zeta<R, L>(nrow, (const C*)U, alpha, (const C*)S, (const C*)Z, (const C*)V, zb, (C*)Rv, (C*)P,
                          (cx<double>*)X, part);
    });
}

template <typename R>
static void convert(int to_internal, long long nsite, int L, const void* in, void* out) {
  const int grid = (int)((nsite * L + NT - 1) / NT);
  if (to_internal)
    emu_launch(grid, 1, NT, 0, [&] { k_abi_to_internal<R>(nsite, L, (const cx<double>*)in, (cx<R>*)out); });
  else
    emu_launch(grid, 1, NT, 0, [&] { k_internal_to_abi<R>(nsite, L, (const cx<R>*)in, (cx<double>*)out); });
}

extern "C" {
// ABI [site][12][rhs] FP64 <-> internal [site][rhs][12] in FP64 or FP32
void emu_convert(int fp64, int to_internal, long long nsite, int L, const void* in, void* out) {
  if (fp64) convert<double>(to_internal, nsite, L, in, out);
  else convert<float>(to_internal, nsite, L, in, out);
}
int emu_convert_links(long long nlinks, const double* in, double* l64, float* l32) {
  int bad = 0;
  emu_launch(3, 1, NT, 0, [&] {
    k_convert_links(nlinks, (const cx<double>*)in, (cx<double>*)l64, (cx<float>*)l32, &bad);
  });
  return bad;
}
void emu_residual_from(int fp64, long long nsite, int L, const double* B, const double* W, void* out, double* part,
                       int ncta) {
  if (fp64)
    emu_launch(ncta, 1, NT, 0, [&] {
      k_residual_from<double>(nsite, L, (const cx<double>*)B, (const cx<double>*)W, (cx<double>*)out, part);
    });
  else
    emu_launch(ncta, 1, NT, 0, [&] {
      k_residual_from<float>(nsite, L, (const cx<double>*)B, (const cx<double>*)W, (cx<float>*)out, part);
    });
}
int emu_abi_check(long long nrow, int L, const double* in, double* part, int ncta) {
  int bad = 0;
  emu_launch(ncta, 1, NT, 0, [&] { k_abi_check(nrow, L, (const cx<double>*)in, part, &bad); });
  return bad;
}
void emu_pack_dummies(long long nrow, int L, int Lt, const double* in, double* out, unsigned long long seed,
                      int random) {
  emu_launch(3, 1, NT, 0, [&] {
    k_pack_dummies(nrow, L, Lt, (const cx<double>*)in, (cx<double>*)out, seed, random);
  });
}
void emu_first_columns(long long nrow, int Lt, int L, const double* in, double* out) {
  emu_launch(3, 1, NT, 0, [&] { k_first_columns(nrow, Lt, L, (const cx<double>*)in, (cx<double>*)out); });
}
int emu_lxl_alpha(int L, const double* part, int nparts, double* G, double* LU, int* piv, double* alpha) {
  int status = 0;
  one_cta(256, [&] { k_lxl_alpha(L, part, nparts, G, LU, piv, alpha, &status); });
  return status;
}
int emu_lxl_zeta_beta(int L, const double* part, int nparts, const double* LU, const int* piv, double* zb,
                      int status_in) {
  int status = status_in;
  one_cta(256, [&] { k_lxl_zeta_beta(L, part, nparts, LU, piv, zb, &status); });
  return status;
}
int emu_lxl_chol(int L, const double* part, int nparts, double* M, double rel_eps, double shift) {
  int status = 0;
  one_cta(256, [&] { k_lxl_chol(L, part, nparts, M, &status, rel_eps, shift); });
  return status;
}
// returns the number of CTAs (partials), or minus the error bits
int emu_gram(int fp64, int L, long long nsite, const void* A, const void* B1, const void* B2, int flags,
             double* part) {
#define G(LL) \
  case LL: return fp64 ? gram<double, LL>(nsite, A, B1, B2, flags, part) : gram<float, LL>(nsite, A, B1, B2, flags, part);
  switch (L) {
    G(3)
    G(4)
    G(5)
    G(12)
  }
#undef G
  return 0;
}
// which: 0 Y = X M (X in U), 1 R -= V alpha, 2 the zeta update (X in FP64)
int emu_updates(int fp64, int L, int which, int ncta, int nrow, const void* U, const double* alpha, const void* S,
                const void* Z, const void* V, const double* zb, void* Rv, void* P, void* X64, double* part,
                const double* M, void* Y) {
#define U_(LL)                                                                                                  \
  case LL:                                                                                                     \
    if (fp64) updates<double, LL>(which, ncta, nrow, U, alpha, S, Z, V, zb, Rv, P, X64, part, M, Y);           \
    else updates<float, LL>(which, ncta, nrow, U, alpha, S, Z, V, zb, Rv, P, X64, part, M, Y);                 \
    return 0;
  switch (L) {
    U_(3)
    U_(4)
    U_(5)
    U_(12)
  }
#undef U_
  return -1;
}
}
