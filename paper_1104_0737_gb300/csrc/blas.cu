// blas.cu — block linear algebra of Algorithm 2 (Sec. 2.1) on N x L blocks in
// the site-major internal layout [site][rhs][spin*3+colour]:
//   - fused block inner products (R~^H V, R~^H R; R~^H Z with Tr(Z^H R) and
//     Tr(Z^H Z); P^H P for the QR) with per-CTA partial sums on a fixed grid,
//     so every reduction is formed in one fixed order (bitwise reproducible);
//   - block AXPYs (the updates of R, X and P) and the QR transform P <- P M;
//   - layout and precision conversions at the ABI boundary;
//   - the L x L algebra (LU with partial pivoting, Cholesky, triangular
//     inverse) in FP64 in single-CTA kernels, so nothing leaves the device
//     inside an iteration but the residual norms.
// FP32 blocks: products in FP32, running sums as TwoSum pairs of FP32, the
// per-CTA partial sums in FP64.
#include <math.h>

#include "internal.h"

namespace mbicg {

namespace {

constexpr int NT = 256;  // threads of the row kernels and the gram kernel

// register block of the gram kernel: BB x BB entries per thread
__host__ __device__ constexpr int reg_block(int L) { return L % 3 == 0 ? 3 : (L % 2 == 0 ? 2 : 1); }
// sites per shared-memory tile of the gram kernel
__host__ __device__ constexpr int gram_tile_sites(int L, int real_bytes) {
  return L >= 8 ? (real_bytes == 4 ? 16 : 8) : (L >= 4 ? 16 : 32);
}

// ---------------------------------------------------------------------------
// Gram kernel
//
// A persistent grid of GRAM_CTAS CTAs walks over tiles of TS sites.  One
// thread streams each tile of every input block into shared memory with bulk
// asynchronous copies (TMA) completing on an mbarrier, STAGES tiles ahead, while
// all threads multiply the tile already in shared memory: thread (lane, block)
// accumulates a BB x BB block of the L x L product over the tile rows
// lane, lane + LANES, ...  With HERM (A^H A), only the blocks on or above the
// diagonal are formed and the rest is mirrored.
// ---------------------------------------------------------------------------
// flags: bit0 G1 = A^H B1, bit1 G2 = A^H B2, bit2 diag(B1^H B2), bit3 diag(B1^H B1)
template <typename R, int L, bool HERM>
struct GramShape {
  static constexpr int BB = reg_block(L);
  static constexpr int NBI = L / BB;
  static constexpr int NB = HERM ? NBI * (NBI + 1) / 2 : NBI * NBI;
  static constexpr int LANES = NT / NB > 0 ? NT / NB : 1;
  static constexpr int TS = gram_tile_sites(L, (int)sizeof(R));
  static constexpr int TILE = TS * L * 12;  // complex numbers per tile per array
  // A^H A streams one array: six stages of it in the room of two stages of
  // three arrays, so that more tiles are in flight per CTA
  static constexpr int NARR = HERM ? 1 : 3;
  static constexpr int STAGES = HERM ? 6 : 2;
  static constexpr size_t tile_bytes = sizeof(cx<R>) * (size_t)TILE;
  static constexpr size_t red_g = sizeof(cx<double>) * LANES * L * L;
  static constexpr size_t red_d = sizeof(cx<double>) * 2 * (NT / L) * L;
  static constexpr size_t stage_area = tile_bytes * NARR * STAGES;
  static constexpr size_t red_bytes = red_g > red_d ? red_g : red_d;
  static constexpr size_t smem = (stage_area > red_bytes ? stage_area : red_bytes) + 64;
};

// Running sums of the Gram kernel's per-tile partial sums.  FP32 blocks: a
// pair of floats, each addition error-free by Knuth's TwoSum (the rounding
// error of hi + a is carried in lo), about 48 significant bits — what FP64
// running sums gave, without FP64 arithmetic, which runs at 1/64 of the FP32
// rate here and, done by every thread at once, stalled the kernel.  FP64
// blocks: one double.
template <typename R>
struct RunSum;
template <>
struct RunSum<double> {
  double v = 0;
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct RunSum<float> {
  float hi = 0, lo = 0;
  __device__ __forceinline__ void add(float a) {
    const float s = hi + a;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (a - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename R, int L, bool HERM>
__global__ void __launch_bounds__(NT, 2) k_gram(long long nsite, const cx<R>* __restrict__ A,
                                             const cx<R>* __restrict__ B1, const cx<R>* __restrict__ B2,
                                             int flags, double* __restrict__ part, int* __restrict__ err) {
  using SH = GramShape<R, L, HERM>;
  constexpr int BB = SH::BB, NBI = SH::NBI, NB = SH::NB, LANES = SH::LANES, TS = SH::TS, TILE = SH::TILE;
  constexpr int STAGES = SH::STAGES, NARR = SH::NARR;
  static_assert(STAGES * sizeof(uint64_t) <= 64, "the stages' mbarriers live in the last 64 bytes");
  // FP32 accumulators collect FLUSH tiles, then go into the running sums
  // (TwoSum pairs); FP64 accumulators go in after every tile
  constexpr int FLUSH = sizeof(R) == 4 ? 8 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (SH::smem - 64));
  cx<R>* stage0 = reinterpret_cast<cx<R>*>(smem_raw);

  const bool g1 = flags & 1, g2 = flags & 2, d1 = flags & 4, d2 = flags & 8;
  // HERM: A = B1 and G1 alone (the launcher's choice), one array per stage
  const bool a_is_b1 = HERM || (A == B1);
  const bool loadA = g1 || g2 || a_is_b1;
  const bool loadB1 = !a_is_b1;
  const bool loadB2 = !HERM && B2 != nullptr;
  const int tid = threadIdx.x;
  const int blk = tid % NB;
  const int lane = tid / NB;
  const bool gram_thread = lane < LANES;
  // block coordinates (on and above the diagonal when HERM)
  int bi, bj;
  if (HERM) {
    int r = 0, rem = blk;
    while (rem >= NBI - r) { rem -= NBI - r; ++r; }
    bi = r * BB;
    bj = (r + rem) * BB;
  } else {
    bi = (blk / NBI) * BB;
    bj = (blk % NBI) * BB;
  }

  cx<R> acc1[BB][BB], acc2[BB][BB];
  RunSum<R> tot1[BB][BB][2], tot2[BB][BB][2];  // [re, im]
#pragma unroll
  for (int i = 0; i < BB; ++i)
#pragma unroll
    for (int j = 0; j < BB; ++j) {
      acc1[i][j] = acc2[i][j] = mk<R>(0, 0);
    }
  const int dcol = tid % L, dlane = tid / L;
  constexpr int DLANES = NT / L;
  cx<R> dacc1 = mk<R>(0, 0);
  R dacc2 = 0;
  RunSum<R> dtot1[2], dtot2;

  const long long ntiles = (nsite + TS - 1) / TS;
  const int my_tiles = (int)(ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int j) {  // tile j of this CTA into stage j % STAGES (thread 0)
    const long long tile = blockIdx.x + (long long)j * gridDim.x;
    const long long site0 = tile * TS;
    const int ns = (int)min((long long)TS, nsite - site0);
    const uint32_t bytes = (uint32_t)(sizeof(cx<R>) * (size_t)ns * L * 12);
    const int st = j % STAGES;
    cx<R>* dst = stage0 + (size_t)st * NARR * TILE;
    const uint32_t total = bytes * ((loadA ? 1 : 0) + (loadB1 ? 1 : 0) + (loadB2 ? 1 : 0));
    mbar_arrive_expect_tx(&bars[st], total);
    const size_t off = (size_t)site0 * L * 12;
    if (loadA) bulk_g2s(dst, A + off, bytes, &bars[st]);
    if (loadB1) bulk_g2s(dst + TILE, B1 + off, bytes, &bars[st]);
    if (loadB2) bulk_g2s(dst + 2 * TILE, B2 + off, bytes, &bars[st]);
  };
  if (tid == 0)
    for (int j = 0; j < STAGES && j < my_tiles; ++j) issue(j);

  bool ok = true;
  int since_flush = 0;
  int j = 0;
  for (; j < my_tiles; ++j) {
    const int st = j % STAGES;
    // a wait that gives up is acted on below, by all threads together
    const bool arrived = mbar_wait_bounded(&bars[st], (uint32_t)((j / STAGES) & 1));
    const long long site0 = (blockIdx.x + (long long)j * gridDim.x) * TS;
    const int ns = (int)min((long long)TS, nsite - site0);
    const cx<R>* sA = stage0 + (size_t)st * NARR * TILE;
    const cx<R>* tB1 = a_is_b1 ? sA : sA + TILE;
    const cx<R>* sB2 = sA + 2 * TILE;
    const int nrows = ns * 12;
    if ((g1 || g2) && gram_thread) {
      for (int row = lane; row < nrows; row += LANES) {
        const int site = row / 12, sc = row - site * 12;
        const cx<R>* ra = sA + site * L * 12 + sc;
        cx<R> a[BB];
#pragma unroll
        for (int i = 0; i < BB; ++i) a[i] = ra[(bi + i) * 12];
        if (g1) {
          const cx<R>* rb = tB1 + site * L * 12 + sc;
#pragma unroll
          for (int jj = 0; jj < BB; ++jj) {
            const cx<R> bv = rb[(bj + jj) * 12];
#pragma unroll
            for (int i = 0; i < BB; ++i) cmac_conj(acc1[i][jj], a[i], bv);
          }
        }
        if (g2) {
          const cx<R>* rb = sB2 + site * L * 12 + sc;
#pragma unroll
          for (int jj = 0; jj < BB; ++jj) {
            const cx<R> bv = rb[(bj + jj) * 12];
#pragma unroll
            for (int i = 0; i < BB; ++i) cmac_conj(acc2[i][jj], a[i], bv);
          }
        }
      }
    }
    if ((d1 || d2) && dlane < DLANES) {
      for (int row = dlane; row < nrows; row += DLANES) {
        const int site = row / 12, sc = row - site * 12;
        const cx<R> z = tB1[(site * L + dcol) * 12 + sc];
        if (d1) cmac_conj(dacc1, z, sB2[(site * L + dcol) * 12 + sc]);
        if (d2) dacc2 = fma(z.re, z.re, fma(z.im, z.im, dacc2));
      }
    }
    if (++since_flush == FLUSH) {
      since_flush = 0;
#pragma unroll
      for (int i = 0; i < BB; ++i)
#pragma unroll
        for (int jj = 0; jj < BB; ++jj) {
          tot1[i][jj][0].add(acc1[i][jj].re); tot1[i][jj][1].add(acc1[i][jj].im);
          tot2[i][jj][0].add(acc2[i][jj].re); tot2[i][jj][1].add(acc2[i][jj].im);
          acc1[i][jj] = acc2[i][jj] = mk<R>(0, 0);
        }
      dtot1[0].add(dacc1.re); dtot1[1].add(dacc1.im); dtot2.add(dacc2);
      dacc1 = mk<R>(0, 0);
      dacc2 = 0;
    }
    if (__syncthreads_or(!arrived)) {  // every thread is done with this stage
      ok = false;
      break;
    }
    if (tid == 0 && j + STAGES < my_tiles) issue(j + STAGES);
  }
  if (!ok) {
    // a copy never completed: record it, and wait (bounded) for the copies
    // still in flight before the shared memory is released
    if (tid == 0) {
      atomicOr(err, ST_TIMEOUT);
      for (int jj = j; jj < my_tiles && jj < j + STAGES; ++jj)
        mbar_wait_bounded(&bars[jj % STAGES], (uint32_t)((jj / STAGES) & 1));
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int i = 0; i < BB; ++i)
#pragma unroll
    for (int jj = 0; jj < BB; ++jj) {
      tot1[i][jj][0].add(acc1[i][jj].re); tot1[i][jj][1].add(acc1[i][jj].im);
      tot2[i][jj][0].add(acc2[i][jj].re); tot2[i][jj][1].add(acc2[i][jj].im);
    }
  dtot1[0].add(dacc1.re); dtot1[1].add(dacc1.im); dtot2.add(dacc2);

  // reduce over lanes through shared memory, fixed order
  __syncthreads();
  cx<double>* red = reinterpret_cast<cx<double>*>(smem_raw);
  const int nslots = 2 * L * L + 2 * L;
  double* out = part + (long long)blockIdx.x * nslots * 2;
  for (int pass = 0; pass < 2; ++pass) {
    const bool on = pass == 0 ? g1 : g2;
    if (!on) {
      for (int e = tid; e < L * L; e += NT) {
        out[(pass * L * L + e) * 2] = 0;
        out[(pass * L * L + e) * 2 + 1] = 0;
      }
      continue;
    }
    if (gram_thread) {
#pragma unroll
      for (int i = 0; i < BB; ++i)
#pragma unroll
        for (int jj = 0; jj < BB; ++jj)
          red[lane * L * L + (bi + i) * L + (bj + jj)] =
              pass == 0 ? mk(tot1[i][jj][0].value(), tot1[i][jj][1].value())
                        : mk(tot2[i][jj][0].value(), tot2[i][jj][1].value());
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += NT) {
      int ei = e / L, ej = e % L;
      bool mirror = false;
      if (HERM && (ei / BB) > (ej / BB)) {  // below the block diagonal: mirror
        const int t = ei; ei = ej; ej = t;
        mirror = true;
      }
      double re = 0, im = 0;
      for (int l = 0; l < LANES; ++l) {
        re += red[l * L * L + ei * L + ej].re;
        im += red[l * L * L + ei * L + ej].im;
      }
      out[(pass * L * L + e) * 2] = re;
      out[(pass * L * L + e) * 2 + 1] = mirror ? -im : im;
    }
    __syncthreads();
  }
  if (dlane < DLANES) {
    red[dlane * L + dcol] = mk(dtot1[0].value(), dtot1[1].value());
    red[DLANES * L + dlane * L + dcol] = mk(dtot2.value(), 0.0);
  }
  __syncthreads();
  for (int e = tid; e < 2 * L; e += NT) {
    const int which = e / L, col = e % L;
    double re = 0, im = 0;
    for (int l = 0; l < DLANES; ++l) {
      re += red[which * DLANES * L + l * L + col].re;
      im += red[which * DLANES * L + l * L + col].im;
    }
    const bool on = which == 0 ? d1 : d2;
    out[(2 * L * L + e) * 2] = on ? re : 0.0;
    out[(2 * L * L + e) * 2 + 1] = on ? im : 0.0;
  }
}

template <typename R, int L, bool HERM>
int launch_gram_t(const Exec& ex, long long nsite, const cx<R>* A, const cx<R>* B1, const cx<R>* B2, int flags,
                  double* part, int* err) {
  using SH = GramShape<R, L, HERM>;
  static const cudaError_t attr_set =  // once per process, thread-safely
      cudaFuncSetAttribute(k_gram<R, L, HERM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::smem);
  (void)attr_set;
  const long long ntiles = (nsite + SH::TS - 1) / SH::TS;
  const int grid = (int)(ntiles < GRAM_CTAS ? ntiles : GRAM_CTAS);
  k_gram<R, L, HERM><<<grid, NT, SH::smem, ex.stream>>>(nsite, A, B1, B2, flags, part, err);
  ++*ex.launches;
  return grid;
}

template <typename R, int L>
int launch_gram(const Exec& ex, long long nsite, const cx<R>* A, const cx<R>* B1, const cx<R>* B2, int flags,
                double* part, int* err) {
  if (!A) A = B1;
  // A^H A alone: Hermitian, only the upper block triangle is formed
  if (A == B1 && flags == GRAM_G1) return launch_gram_t<R, L, true>(ex, nsite, A, B1, B2, flags, part, err);
  return launch_gram_t<R, L, false>(ex, nsite, A, B1, B2, flags, part, err);
}

// ---------------------------------------------------------------------------
// row kernels: one thread per row (site, spin*3+colour), L columns in registers
// ---------------------------------------------------------------------------
// rows (site, spin*3+colour) are below 2^31 (volume <= 2^27 sites)
__device__ __forceinline__ size_t row_base(int row, int L) {
  const int site = (unsigned)row / 12u;
  return (size_t)site * L * 12 + (row - site * 12);
}

// The loops over output columns stay rolled in both precisions: unrolled
// (fully, or by 2 or 4) the FP32 update kernels grew from 48-64 to 102-255
// registers per thread, spilling when fully unrolled, while their rolled
// form already reaches 66-91 % of HBM.
template <typename R, int L>
__host__ __device__ constexpr int col_unroll() { return 1; }

template <typename R, int L>
__global__ void __launch_bounds__(NT) k_transform(int nrow, const cx<R>* X, const double* __restrict__ M,
                                                  cx<R>* Y) {
  __shared__ cx<R> sM[L * L];
  for (int e = threadIdx.x; e < L * L; e += NT) sM[e] = mk((R)M[2 * e], (R)M[2 * e + 1]);
  __syncthreads();
  for (int row = blockIdx.x * NT + threadIdx.x; row < nrow; row += gridDim.x * NT) {
    const size_t b = row_base(row, L);
    cx<R> x[L];
#pragma unroll
    for (int k = 0; k < L; ++k) x[k] = X[b + k * 12];
#pragma unroll(col_unroll<R, L>())
    for (int j = 0; j < L; ++j) {
      cx<R> y = mk<R>(0, 0);
#pragma unroll
      for (int k = 0; k < L; ++k) cmac(y, x[k], sM[k * L + j]);
      Y[b + j * 12] = y;
    }
  }
}

// R -= V alpha; X += U alpha is deferred to k_update_zeta
template <typename R, int L>
__global__ void __launch_bounds__(NT) k_update_alpha(int nrow, const cx<R>* __restrict__ V,
                                                     const double* __restrict__ alpha, cx<R>* __restrict__ Rv) {
  __shared__ cx<R> sA[L * L];
  for (int e = threadIdx.x; e < L * L; e += NT) sA[e] = mk((R)alpha[2 * e], (R)alpha[2 * e + 1]);
  __syncthreads();
  for (int row = blockIdx.x * NT + threadIdx.x; row < nrow; row += gridDim.x * NT) {
    const size_t b = row_base(row, L);
    cx<R> v[L];
#pragma unroll
    for (int k = 0; k < L; ++k) v[k] = V[b + k * 12];
#pragma unroll(col_unroll<R, L>())
    for (int j = 0; j < L; ++j) {
      cx<R> va = mk<R>(0, 0);
#pragma unroll
      for (int k = 0; k < L; ++k) cmac(va, v[k], sA[k * L + j]);
      Rv[b + j * 12] = Rv[b + j * 12] - va;
    }
  }
}

// X += U alpha + zeta S (one update in Algorithm 1, which Algorithm 2 splits
// into its U alpha and zeta S parts), R -= zeta Z, P = R + (P - zeta V) beta,
// and the squared column norms of the new R.  X is accumulated in
// FP64; its increment U alpha + zeta S is formed in the Krylov vectors'
// precision (they are its inputs), so FP32 vectors cost two FP64 adds per
// element rather than FP64 products (FP64 runs at 1/64 of the FP32 rate).
// zb = [zeta, beta (L x L)] complex double
template <typename R, int L>
__global__ void __launch_bounds__(NT) k_update_zeta(int nrow, const cx<R>* __restrict__ U,
                                                    const double* __restrict__ alpha, const cx<R>* __restrict__ S,
                                                    const cx<R>* __restrict__ Z, const cx<R>* __restrict__ V,
                                                    const double* __restrict__ zb, cx<R>* __restrict__ Rv,
                                                    cx<R>* __restrict__ P, cx<double>* __restrict__ X64,
                                                    double* __restrict__ part) {
  __shared__ cx<R> sB[L * L];
  __shared__ cx<R> sA[L * L];
  __shared__ double sred[NT];
  for (int e = threadIdx.x; e < L * L; e += NT) {
    sB[e] = mk((R)zb[2 + 2 * e], (R)zb[3 + 2 * e]);
    sA[e] = mk((R)alpha[2 * e], (R)alpha[2 * e + 1]);
  }
  const cx<R> zeta = mk((R)zb[0], (R)zb[1]);
  __syncthreads();
  R nrm[L];
#pragma unroll
  for (int j = 0; j < L; ++j) nrm[j] = 0;
  for (int row = blockIdx.x * NT + threadIdx.x; row < nrow; row += gridDim.x * NT) {
    const size_t b = row_base(row, L);
    cx<R> t[L];
    {
      cx<R> u[L];
#pragma unroll
      for (int k = 0; k < L; ++k) u[k] = U[b + k * 12];
#pragma unroll(col_unroll<R, L>())
      for (int j = 0; j < L; ++j) {
        cx<R> ua = mk<R>(0, 0);
#pragma unroll
        for (int k = 0; k < L; ++k) cmac(ua, u[k], sA[k * L + j]);
        const cx<R> s = S[b + j * 12];
        const R dre = ua.re + (zeta.re * s.re - zeta.im * s.im);
        const R dim = ua.im + (zeta.re * s.im + zeta.im * s.re);
        cx<double> x = X64[b + j * 12];
        x.re += (double)dre;
        x.im += (double)dim;
        X64[b + j * 12] = x;
      }
    }
#pragma unroll
    for (int k = 0; k < L; ++k) {
      const cx<R> rn = Rv[b + k * 12] - zeta * Z[b + k * 12];
      Rv[b + k * 12] = rn;
      nrm[k] = fma(rn.re, rn.re, fma(rn.im, rn.im, nrm[k]));
      t[k] = P[b + k * 12] - zeta * V[b + k * 12];
    }
#pragma unroll(col_unroll<R, L>())
    for (int j = 0; j < L; ++j) {
      cx<R> y = Rv[b + j * 12];  // the new R, just written
#pragma unroll
      for (int k = 0; k < L; ++k) cmac(y, t[k], sB[k * L + j]);
      P[b + j * 12] = y;
    }
  }
  // column norms: reduce over the CTA
#pragma unroll
  for (int j = 0; j < L; ++j) {
    sred[threadIdx.x] = (double)nrm[j];
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) sred[threadIdx.x] += sred[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.x * L + j] = sred[0];
    __syncthreads();
  }
}

// dst (device memory) = src (registered host memory, read through its mapped
// device address), n 16-byte words.  Every thread keeps four loads in flight,
// so the host pages are fetched by the whole grid at once rather than by one
// copy engine in sequence.
__global__ void __launch_bounds__(NT) k_copy_mapped(long long n, const uint4* src, uint4* __restrict__ dst) {
  const long long stride = (long long)gridDim.x * NT;
  long long i = blockIdx.x * (long long)NT + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n; i += stride) dst[i] = src[i];
}

// The first two rows of every FP32 link: [site][mu][9] -> [site][mu][6]
__global__ void __launch_bounds__(NT) k_links_to_rows(long long n, const cx<float>* __restrict__ U,
                                                      cx<float>* __restrict__ R) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const long long l = i / 6, k = i - l * 6;
    R[i] = U[l * 9 + k];
  }
}

// Columns of an ABI block (rows [site][spin*colour], L columns) copied into
// the first L of Lt columns, the other Lt - L filled with Gaussian random
// numbers (or zeros): a counter-based generator, splitmix64 of (seed, row,
// column) giving two uniforms, and the Box-Muller transform.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_pack_dummies(long long nrow, int L, int Lt, const cx<double>* __restrict__ in,
                               cx<double>* __restrict__ out, unsigned long long seed, int random) {
  const long long n = nrow * Lt;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / Lt;
    const int j = (int)(i - row * Lt);
    if (j < L) {
      out[i] = in[row * L + j];
    } else if (random) {
      const unsigned long long h1 = splitmix64(seed ^ splitmix64((unsigned long long)i));
      const unsigned long long h2 = splitmix64(h1);
      const double u1 = ((double)(h1 >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
      const double u2 = (double)(h2 >> 11) * 0x1.0p-53;          // [0, 1)
      const double rad = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      out[i] = mk(rad * cs, rad * sn);
    } else {
      out[i] = mk(0.0, 0.0);
    }
  }
}
// the first L of Lt columns
__global__ void k_first_columns(long long nrow, int Lt, int L, const cx<double>* __restrict__ in,
                                cx<double>* __restrict__ out) {
  const long long n = nrow * L;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / L;
    out[i] = in[row * Lt + (i - row * L)];
  }
}

int row_grid(long long nrow) {
  const long long need = (nrow + NT - 1) / NT;
  return (int)(need < 8 * 152 ? need : 8 * 152);
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_abi_to_internal(long long nsite, int L, const cx<double>* __restrict__ in, cx<R>* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // site * L + rhs
  if (idx >= nsite * L) return;
  const int site = idx / L;
  const int rhs = idx - site * L;
#pragma unroll
  for (int sc = 0; sc < 12; ++sc) {
    const cx<double> v = in[((size_t)site * 12 + sc) * L + rhs];
    out[(size_t)idx * 12 + sc] = mk((R)v.re, (R)v.im);
  }
}
template <typename R>
__global__ void k_internal_to_abi(long long nsite, int L, const cx<R>* __restrict__ in, cx<double>* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsite * L) return;
  const int site = idx / L;
  const int rhs = idx - site * L;
#pragma unroll
  for (int sc = 0; sc < 12; ++sc) {
    const cx<R> v = in[(size_t)idx * 12 + sc];
    out[((size_t)site * 12 + sc) * L + rhs] = mk((double)v.re, (double)v.im);
  }
}
template <typename RI, typename RO>
__global__ void k_convert(long long n, const cx<RI>* __restrict__ in, cx<RO>* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = mk((RO)in[i].re, (RO)in[i].im);
}
// copies and converts the links, flags NaN/Inf (bit 0) and links that are
// not SU(3) to 1e-10 (bit 1: U U^dagger != 1 or det U != 1)
__global__ void k_convert_links(long long nlinks, const cx<double>* __restrict__ in, cx<double>* __restrict__ l64,
                                cx<float>* __restrict__ l32, int* bad) {
  for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks;
       l += (long long)gridDim.x * blockDim.x) {
    cx<double> u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      u[e] = in[l * 9 + e];
      if (!isfinite(u[e].re) || !isfinite(u[e].im)) atomicOr(bad, 1);
      l64[l * 9 + e] = u[e];
      l32[l * 9 + e] = mk((float)u[e].re, (float)u[e].im);
    }
    double dev = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double re = (i == j) ? -1.0 : 0.0, im = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {  // (U U^dagger)_ij = sum_k U_ik conj(U_jk)
          const cx<double> a = u[i * 3 + k], b = u[j * 3 + k];
          re += a.re * b.re + a.im * b.im;
          im += a.im * b.re - a.re * b.im;
        }
        dev = fmax(dev, fabs(re) + fabs(im));
      }
    // det U = u0 (u4 u8 - u5 u7) - u1 (u3 u8 - u5 u6) + u2 (u3 u7 - u4 u6)
    auto mul = [](cx<double> a, cx<double> b) { return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); };
    auto sub = [](cx<double> a, cx<double> b) { return mk(a.re - b.re, a.im - b.im); };
    const cx<double> m0 = sub(mul(u[4], u[8]), mul(u[5], u[7]));
    const cx<double> m1 = sub(mul(u[3], u[8]), mul(u[5], u[6]));
    const cx<double> m2 = sub(mul(u[3], u[7]), mul(u[4], u[6]));
    const cx<double> det = sub(mul(u[0], m0), sub(mul(u[1], m1), mul(u[2], m2)));
    dev = fmax(dev, fabs(det.re - 1.0) + fabs(det.im));
    if (!(dev <= 1e-10)) atomicOr(bad, 2);
  }
}

// out = B - W (internal layout) in R, per-CTA column norms (thread rhs fixed)
template <typename R>
__global__ void __launch_bounds__(NT) k_residual_from(long long nsite, int L, const cx<double>* __restrict__ B,
                                                     const cx<double>* __restrict__ W, cx<R>* __restrict__ out,
                                                     double* __restrict__ part) {
  __shared__ double sred[NT];
  const int per = (NT / L) * L;  // threads used: a multiple of L, so rhs is fixed per thread
  const int tid = threadIdx.x;
  double acc = 0;
  if (tid < per) {
    const long long stride = (long long)gridDim.x * per;
    for (long long idx = (long long)blockIdx.x * per + tid; idx < nsite * L; idx += stride) {
#pragma unroll
      for (int sc = 0; sc < 12; ++sc) {
        const cx<double> b = B[idx * 12 + sc];
        const cx<double> w = W ? W[idx * 12 + sc] : mk(0.0, 0.0);
        const cx<double> r = mk(b.re - w.re, b.im - w.im);
        out[idx * 12 + sc] = mk((R)r.re, (R)r.im);
        acc += r.re * r.re + r.im * r.im;
      }
    }
  }
  sred[tid] = acc;
  __syncthreads();
  if (tid < L) {
    double s = 0;
    for (int t = tid; t < per; t += L) s += sred[t];
    part[(long long)blockIdx.x * L + tid] = s;
  }
}

// NaN/Inf scan and column norms of an ABI-layout block ([row][rhs], row = site*12+sc)
__global__ void __launch_bounds__(NT) k_abi_check(long long nrow, int L, const cx<double>* __restrict__ in,
                                                 double* __restrict__ part, int* bad) {
  __shared__ double sred[NT];
  const int per = (NT / L) * L;
  const int tid = threadIdx.x;
  double acc = 0;
  if (tid < per) {
    const long long stride = (long long)gridDim.x * per;
    for (long long idx = (long long)blockIdx.x * per + tid; idx < nrow * L; idx += stride) {
      const cx<double> v = in[idx];
      if (!isfinite(v.re) || !isfinite(v.im)) atomicOr(bad, 1);
      acc += v.re * v.re + v.im * v.im;
    }
  }
  sred[tid] = acc;
  __syncthreads();
  if (tid < L) {
    double s = 0;
    for (int t = tid; t < per; t += L) s += sred[t];
    part[(long long)blockIdx.x * L + tid] = s;
  }
}

// ---------------------------------------------------------------------------
// L x L algebra (FP64, one CTA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b) {
  const double d = b.re * b.re + b.im * b.im;
  return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__device__ __forceinline__ double cabs2(cx<double> a) { return a.re * a.re + a.im * a.im; }

// sum partials: dst[e] = sum_p part[p][slot0 + e], e < count (complex)
__device__ void reduce_slots(const double* part, int nparts, int nslots, int slot0, int count, cx<double>* dst) {
  for (int e = threadIdx.x; e < count; e += blockDim.x) {
    double re = 0, im = 0;
    for (int p = 0; p < nparts; ++p) {
      re += part[((long long)p * nslots + slot0 + e) * 2];
      im += part[((long long)p * nslots + slot0 + e) * 2 + 1];
    }
    dst[e] = mk(re, im);
  }
}

// The L x L kernels run in one CTA.  The factorisations proceed column by
// column with the work of a step spread over the threads (rows, matrix
// entries or right-hand-side columns); every entry is computed by the same
// expression, with the same operands in the same order, as in a sequential
// loop, so the result does not depend on the thread count.
__device__ __forceinline__ cx<double> csub_mul(cx<double> s, cx<double> f, cx<double> a) {  // s - f a
  return mk(s.re - (f.re * a.re - f.im * a.im), s.im - (f.re * a.im + f.im * a.re));
}

__global__ void k_lxl_alpha(int L, const double* part, int nparts, double* G, double* LU, int* piv, double* alpha,
                            int* status) {
  __shared__ cx<double> sG[MAXL * MAXL], sC[MAXL * MAXL];
  __shared__ double smax[256];
  __shared__ int s_st, s_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nslots = 2 * L * L + 2 * L;
  reduce_slots(part, nparts, nslots, 0, L * L, sG);
  reduce_slots(part, nparts, nslots, L * L, L * L, sC);
  __syncthreads();
  double m = 0;
  for (int e = tid; e < L * L; e += nt) {
    G[2 * e] = sG[e].re;
    G[2 * e + 1] = sG[e].im;
    m = fmax(m, sqrt(cabs2(sG[e])));
  }
  smax[tid] = m;
  __syncthreads();
  if (tid == 0) {
    double gmax = 0;
    for (int t = 0; t < nt; ++t) gmax = fmax(gmax, smax[t]);  // max: exact in any order
    smax[0] = gmax;
    s_st = isfinite(gmax) ? 0 : ST_NAN;
  }
  __syncthreads();
  const double gmax = smax[0];
  // LU with partial pivoting; C carried along
  for (int k = 0; k < L; ++k) {
    if (tid == 0 && !s_st) {
      int p = k;
      double best = cabs2(sG[k * L + k]);
      for (int r = k + 1; r < L; ++r)
        if (cabs2(sG[r * L + k]) > best) { best = cabs2(sG[r * L + k]); p = r; }
      if (!(sqrt(best) > 1e-300 + 1e-15 * gmax)) s_st |= ST_ALPHA_SINGULAR;
      piv[k] = p;
      s_p = p;
    }
    __syncthreads();
    if (s_st) break;
    const int p = s_p;
    if (p != k)
      for (int c = tid; c < L; c += nt) {
        cx<double> t = sG[k * L + c]; sG[k * L + c] = sG[p * L + c]; sG[p * L + c] = t;
        t = sC[k * L + c]; sC[k * L + c] = sC[p * L + c]; sC[p * L + c] = t;
      }
    __syncthreads();
    for (int r = k + 1 + tid; r < L; r += nt) sG[r * L + k] = cdiv(sG[r * L + k], sG[k * L + k]);  // multipliers
    __syncthreads();
    const int nr = L - 1 - k, ncg = L - 1 - k;
    for (int w = tid; w < nr * (ncg + L); w += nt) {
      const int r = k + 1 + w / (ncg + L), q = w % (ncg + L);
      const cx<double> f = sG[r * L + k];
      if (q < ncg) {
        const int c = k + 1 + q;
        sG[r * L + c] = csub_mul(sG[r * L + c], f, sG[k * L + c]);
      } else {
        const int c = q - ncg;
        sC[r * L + c] = csub_mul(sC[r * L + c], f, sC[k * L + c]);
      }
    }
    __syncthreads();
  }
  const int st = s_st;
  if (!st) {
    // back substitution, one right-hand-side column per thread
    for (int c = tid; c < L; c += nt)
      for (int k = L - 1; k >= 0; --k) {
        cx<double> s = sC[k * L + c];
        for (int j = k + 1; j < L; ++j) s = csub_mul(s, sG[k * L + j], sC[j * L + c]);
        sC[k * L + c] = cdiv(s, sG[k * L + k]);
      }
    __syncthreads();
    for (int e = tid; e < L * L; e += nt) {
      LU[2 * e] = sG[e].re;
      LU[2 * e + 1] = sG[e].im;
      alpha[2 * e] = sC[e].re;
      alpha[2 * e + 1] = sC[e].im;
    }
  } else {
    for (int e = tid; e < 2 * L * L; e += nt) alpha[e] = 0;
  }
  if (tid == 0) *status |= st;
}

__global__ void k_lxl_zeta_beta(int L, const double* part, int nparts, const double* LU, const int* piv, double* zb,
                                int* status) {
  __shared__ cx<double> sC[MAXL * MAXL], sD[2 * MAXL];
  __shared__ int s_st;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nslots = 2 * L * L + 2 * L;
  reduce_slots(part, nparts, nslots, 0, L * L, sC);
  reduce_slots(part, nparts, nslots, 2 * L * L, 2 * L, sD);
  __syncthreads();
  if (tid == 0) {
    int st = *status & ST_ALPHA_SINGULAR;
    cx<double> zr = mk(0.0, 0.0);
    double zz = 0;
    for (int i = 0; i < L; ++i) {
      zr.re += sD[i].re;
      zr.im += sD[i].im;
      zz += sD[L + i].re;
    }
    if (!isfinite(zz) || !isfinite(zr.re) || !isfinite(zr.im)) st |= ST_NAN;
    else if (!(zz > 0)) st |= ST_ZZ_ZERO;
    cx<double> zeta = mk(0.0, 0.0);
    if (!st) zeta = mk(zr.re / zz, zr.im / zz);
    zb[0] = zeta.re;
    zb[1] = zeta.im;
    s_st = st;
  }
  __syncthreads();
  const int st = s_st;
  if (!st) {
    // beta = -(R~^H V)^-1 R~^H Z with the LU factors of the alpha solve, one
    // column per thread: the row interchanges of the factorisation in order
    // (the stored multipliers belong to the final row order), forward
    // substitution with the unit lower factor, back substitution
    for (int c = tid; c < L; c += nt) {
      for (int r = 0; r < L; ++r) sC[r * L + c] = mk(-sC[r * L + c].re, -sC[r * L + c].im);
      for (int k = 0; k < L; ++k) {
        const int p = piv[k];
        if (p != k) { cx<double> t = sC[k * L + c]; sC[k * L + c] = sC[p * L + c]; sC[p * L + c] = t; }
      }
      for (int k = 0; k < L; ++k)
        for (int r = k + 1; r < L; ++r)
          sC[r * L + c] = csub_mul(sC[r * L + c], mk(LU[2 * (r * L + k)], LU[2 * (r * L + k) + 1]), sC[k * L + c]);
      for (int k = L - 1; k >= 0; --k) {
        cx<double> s = sC[k * L + c];
        for (int j = k + 1; j < L; ++j)
          s = csub_mul(s, mk(LU[2 * (k * L + j)], LU[2 * (k * L + j) + 1]), sC[j * L + c]);
        sC[k * L + c] = cdiv(s, mk(LU[2 * (k * L + k)], LU[2 * (k * L + k) + 1]));
      }
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += nt) {
      zb[2 + 2 * e] = sC[e].re;
      zb[3 + 2 * e] = sC[e].im;
    }
  } else {
    for (int e = tid; e < 2 * L * L; e += nt) zb[2 + e] = 0;
  }
  if (tid == 0) *status |= st;
}

// G = gamma^H gamma (gamma upper triangular, real positive diagonal); M = gamma^-1
__global__ void k_lxl_chol(int L, const double* part, int nparts, double* M, int* status, double rel_eps,
                           double shift) {
  __shared__ cx<double> sG[MAXL * MAXL], sR[MAXL * MAXL];
  __shared__ int s_st;
  __shared__ double s_rjj;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nslots = 2 * L * L + 2 * L;
  reduce_slots(part, nparts, nslots, 0, L * L, sG);
  for (int e = tid; e < L * L; e += nt) sR[e] = mk(0.0, 0.0);
  __syncthreads();
  if (tid == 0) {
    if (shift > 0) {
      // shifted factorisation: G + s I with s = shift * max_j G_jj
      double gmax = 0;
      for (int j = 0; j < L; ++j) gmax = fmax(gmax, sG[j * L + j].re);
      for (int j = 0; j < L; ++j) sG[j * L + j].re += shift * gmax;
    }
    s_st = 0;
  }
  __syncthreads();
  for (int j = 0; j < L; ++j) {
    if (tid == 0) {
      double d = sG[j * L + j].re;
      for (int k = 0; k < j; ++k) d -= cabs2(sR[k * L + j]);
      if (!isfinite(d)) s_st |= ST_NAN;
      else if (!(d > rel_eps * sG[j * L + j].re) || !(d > 0)) s_st |= ST_CHOL_FAIL;
      else {
        s_rjj = sqrt(d);
        sR[j * L + j] = mk(s_rjj, 0.0);
      }
    }
    __syncthreads();
    if (s_st) break;
    const double rjj = s_rjj;
    for (int i = j + 1 + tid; i < L; i += nt) {
      // R_ji = (G_ji - sum_k conj(R_kj) R_ki) / R_jj
      cx<double> s = sG[j * L + i];
      for (int k = 0; k < j; ++k) {
        const cx<double> a = sR[k * L + j], b = sR[k * L + i];
        s = mk(s.re - (a.re * b.re + a.im * b.im), s.im - (a.re * b.im - a.im * b.re));
      }
      sR[j * L + i] = mk(s.re / rjj, s.im / rjj);
    }
    __syncthreads();
  }
  const int st = s_st;
  // M = R^-1 (upper triangular), one column per thread: R M = 1
  for (int e = tid; e < L * L; e += nt) sG[e] = mk(0.0, 0.0);
  __syncthreads();
  if (!st) {
    for (int c = tid; c < L; c += nt)
      for (int i = c; i >= 0; --i) {
        cx<double> s = mk(i == c ? 1.0 : 0.0, 0.0);
        for (int k = i + 1; k <= c; ++k) s = csub_mul(s, sR[i * L + k], sG[k * L + c]);
        sG[i * L + c] = mk(s.re / sR[i * L + i].re, s.im / sR[i * L + i].re);
      }
  } else {
    for (int i = tid; i < L; i += nt) sG[i * L + i] = mk(1.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < L * L; e += nt) {
    M[2 * e] = sG[e].re;
    M[2 * e + 1] = sG[e].im;
  }
  if (tid == 0) *status |= st;
}

__global__ void k_lxl_norms(int L, const double* part, int nparts, int from_gram, double* norms, int* status) {
  const int i = threadIdx.x;
  if (i >= L) return;
  double s = 0;
  if (from_gram) {
    const int nslots = 2 * L * L + 2 * L;
    for (int p = 0; p < nparts; ++p) s += part[((long long)p * nslots + 2 * L * L + L + i) * 2];
  } else {
    for (int p = 0; p < nparts; ++p) s += part[(long long)p * L + i];
  }
  norms[i] = s;
  if (!isfinite(s)) atomicOr(status, ST_NAN);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int gram_slots(int L) { return 2 * L * L + 2 * L; }

#define DISPATCH_L(L, CALL)     \
  switch (L) {                  \
    case 1: { constexpr int LL = 1; CALL; } break;   \
    case 2: { constexpr int LL = 2; CALL; } break;   \
    case 3: { constexpr int LL = 3; CALL; } break;   \
    case 4: { constexpr int LL = 4; CALL; } break;   \
    case 5: { constexpr int LL = 5; CALL; } break;   \
    case 6: { constexpr int LL = 6; CALL; } break;   \
    case 7: { constexpr int LL = 7; CALL; } break;   \
    case 8: { constexpr int LL = 8; CALL; } break;   \
    case 9: { constexpr int LL = 9; CALL; } break;   \
    case 10: { constexpr int LL = 10; CALL; } break; \
    case 11: { constexpr int LL = 11; CALL; } break; \
    case 12: { constexpr int LL = 12; CALL; } break; \
    case 13: { constexpr int LL = 13; CALL; } break; \
    case 14: { constexpr int LL = 14; CALL; } break; \
    case 15: { constexpr int LL = 15; CALL; } break; \
    case 16: { constexpr int LL = 16; CALL; } break; \
    default: break;             \
  }

template <typename R>
int block_gram(const Exec& ex, long long nsite, int L, const cx<R>* A, const cx<R>* B1, const cx<R>* B2,
               int flags, double* part, int* err) {
  int grid = -1;
  DISPATCH_L(L, grid = (launch_gram<R, LL>(ex, nsite, A, B1, B2, flags, part, err)));
  return grid;
}

template <typename R>
void block_transform(const Exec& ex, long long nsite, int L, const cx<R>* X, const double* M, cx<R>* Y) {
  const int nrow = (int)(nsite * 12);
  DISPATCH_L(L, (k_transform<R, LL><<<row_grid(nrow), NT, 0, ex.stream>>>(nrow, X, M, Y)));
  ++*ex.launches;
}

template <typename R>
void block_update_alpha(const Exec& ex, long long nsite, int L, const cx<R>* V, const double* alpha, cx<R>* Rv) {
  const int nrow = (int)(nsite * 12);
  DISPATCH_L(L, (k_update_alpha<R, LL><<<row_grid(nrow), NT, 0, ex.stream>>>(nrow, V, alpha, Rv)));
  ++*ex.launches;
}

template <typename R>
int block_update_zeta(const Exec& ex, long long nsite, int L, const cx<R>* U, const double* alpha, const cx<R>* S,
                      const cx<R>* Z, const cx<R>* V, const double* zeta_beta, cx<R>* Rv, cx<R>* P, cx<double>* X64,
                      double* part) {
  const int nrow = (int)(nsite * 12);
  const int grid = row_grid(nrow);
  DISPATCH_L(L, (k_update_zeta<R, LL><<<grid, NT, 0, ex.stream>>>(nrow, U, alpha, S, Z, V, zeta_beta, Rv, P, X64,
                                                                  part)));
  ++*ex.launches;
  return grid;
}

void links_to_rows(const Exec& ex, long long nsite, const cx<float>* U32, cx<float>* U12) {
  const long long n = nsite * 4 * 6;
  k_links_to_rows<<<row_grid(n), NT, 0, ex.stream>>>(n, U32, U12);
  ++*ex.launches;
}

void copy_from_mapped_host(const Exec& ex, const void* src, void* dst, size_t bytes) {
  const long long n = (long long)(bytes / 16);
  k_copy_mapped<<<row_grid(n), NT, 0, ex.stream>>>(n, static_cast<const uint4*>(src), static_cast<uint4*>(dst));
  ++*ex.launches;
}

template <typename R>
void abi_to_internal(const Exec& ex, long long nsite, int L, const cx<double>* in, cx<R>* out) {
  const long long n = nsite * L;
  k_abi_to_internal<R><<<(unsigned)((n + NT - 1) / NT), NT, 0, ex.stream>>>(nsite, L, in, out);
  ++*ex.launches;
}
template <typename R>
void internal_to_abi(const Exec& ex, long long nsite, int L, const cx<R>* in, cx<double>* out) {
  const long long n = nsite * L;
  k_internal_to_abi<R><<<(unsigned)((n + NT - 1) / NT), NT, 0, ex.stream>>>(nsite, L, in, out);
  ++*ex.launches;
}
template <typename RI, typename RO>
void convert_block(const Exec& ex, long long n, const cx<RI>* in, cx<RO>* out) {
  k_convert<RI, RO><<<row_grid(n), NT, 0, ex.stream>>>(n, in, out);
  ++*ex.launches;
}
void pack_dummies(const Exec& ex, long long nsite, int L, int Lt, const cx<double>* in, cx<double>* out,
                  unsigned long long seed, bool random) {
  k_pack_dummies<<<row_grid(nsite * 12 * Lt), NT, 0, ex.stream>>>(nsite * 12, L, Lt, in, out, seed, random ? 1 : 0);
  ++*ex.launches;
}
void first_columns(const Exec& ex, long long nsite, int Lt, int L, const cx<double>* in, cx<double>* out) {
  k_first_columns<<<row_grid(nsite * 12 * L), NT, 0, ex.stream>>>(nsite * 12, Lt, L, in, out);
  ++*ex.launches;
}
void convert_links(const Exec& ex, long long nsite, const cx<double>* in, cx<double>* l64, cx<float>* l32, int* bad) {
  const long long n = nsite * 4;
  k_convert_links<<<row_grid(n), NT, 0, ex.stream>>>(n, in, l64, l32, bad);
  ++*ex.launches;
}
template <typename R>
int residual_from(const Exec& ex, long long nsite, int L, const cx<double>* B64, const cx<double>* W64, cx<R>* out,
                  double* part) {
  const int grid = row_grid(nsite * L);
  k_residual_from<R><<<grid, NT, 0, ex.stream>>>(nsite, L, B64, W64, out, part);
  ++*ex.launches;
  return grid;
}
int abi_check(const Exec& ex, long long n_rows, int L, const cx<double>* in, double* part, int* bad) {
  const int grid = row_grid(n_rows * L);
  k_abi_check<<<grid, NT, 0, ex.stream>>>(n_rows, L, in, part, bad);
  ++*ex.launches;
  return grid;
}

void lxl_alpha(const Exec& ex, int L, const double* part, int nparts, SmallWork& w) {
  k_lxl_alpha<<<1, 256, 0, ex.stream>>>(L, part, nparts, w.G, w.LU, w.piv, w.alpha, w.status);
  ++*ex.launches;
}
void lxl_zeta_beta(const Exec& ex, int L, const double* part, int nparts, SmallWork& w) {
  k_lxl_zeta_beta<<<1, 256, 0, ex.stream>>>(L, part, nparts, w.LU, w.piv, w.zb, w.status);
  ++*ex.launches;
}
void lxl_cholesky_inverse(const Exec& ex, int L, const double* part, int nparts, SmallWork& w, double rel_eps,
                          double shift) {
  k_lxl_chol<<<1, 256, 0, ex.stream>>>(L, part, nparts, w.M, w.status, rel_eps, shift);
  ++*ex.launches;
}
void lxl_norms(const Exec& ex, int L, const double* part, int nparts, bool from_gram, SmallWork& w) {
  k_lxl_norms<<<1, 32, 0, ex.stream>>>(L, part, nparts, from_gram ? 1 : 0, w.norms, w.status);
  ++*ex.launches;
}

__global__ void k_loop_control(LoopCtl* c, const double* __restrict__ norms, const double* __restrict__ bnorm,
                               const int* __restrict__ status, double* __restrict__ hist, int hist_len,
                               cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  double rm = 0;
  for (int i = 0; i < c->Lc; ++i) {
    const double r = sqrt(norms[i]) / bnorm[i];
    if (!(r <= rm)) rm = r;  // a NaN propagates
  }
  c->relmax = rm;
  const int it = c->it + 1;
  if (it - 1 < hist_len) hist[it - 1] = rm;
  c->it = it;
  const bool cont = *status == 0 && rm == rm && rm > c->tol && it < c->max_iter &&
                    !(c->sloppy && rm < c->delta_ru * c->rmax_ru);
  cudaGraphSetConditional(h, cont ? 1u : 0u);
}

void loop_control(const Exec& ex, LoopCtl* ctl, const double* norms, const double* bnorm, const int* status,
                  double* hist, int hist_len, cudaGraphConditionalHandle h) {
  k_loop_control<<<1, 32, 0, ex.stream>>>(ctl, norms, bnorm, status, hist, hist_len, h);
  ++*ex.launches;
}

#define INST(R)                                                                                                   \
  template int block_gram<R>(const Exec&, long long, int, const cx<R>*, const cx<R>*, const cx<R>*, int,        \
                             double*, int*);                                                                      \
  template void block_transform<R>(const Exec&, long long, int, const cx<R>*, const double*, cx<R>*);              \
  template void block_update_alpha<R>(const Exec&, long long, int, const cx<R>*, const double*, cx<R>*);         \
  template int block_update_zeta<R>(const Exec&, long long, int, const cx<R>*, const double*, const cx<R>*,        \
                                    const cx<R>*, const cx<R>*, const double*, cx<R>*, cx<R>*, cx<double>*,       \
                                    double*);                                                                    \
  template void abi_to_internal<R>(const Exec&, long long, int, const cx<double>*, cx<R>*);                        \
  template void internal_to_abi<R>(const Exec&, long long, int, const cx<R>*, cx<double>*);                        \
  template int residual_from<R>(const Exec&, long long, int, const cx<double>*, const cx<double>*, cx<R>*, double*);
INST(float)
INST(double)
#undef INST
template void convert_block<double, float>(const Exec&, long long, const cx<double>*, cx<float>*);
template void convert_block<float, double>(const Exec&, long long, const cx<float>*, cx<double>*);

}  // namespace mbicg
