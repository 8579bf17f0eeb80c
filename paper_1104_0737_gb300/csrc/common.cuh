// common.cuh — complex arithmetic, lattice geometry and the spin projectors of
// the Wilson hopping term (Sec. 2.1, Eq. (hoppingterm)) shared by the kernels.
//
// Internal layouts (device, owned by the library):
//   links   [site][mu][a][b] complex, FP64 and FP32 copies
//   blocks  [site][rhs][spin][colour] complex ("site-major"): the L spinors of
//           a site are contiguous, so one thread per (site, rhs) reads a
//           96-byte (FP32) or 192-byte (FP64) spinor with vector loads and the
//           threads of a warp share the site's links.
// Sites are numbered lexicographically, s = x + Lx*(y + Ly*(z + Lz*t)).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbicg {

// MR steps per domain solve (the sweep keeps a domain's frozen step lengths
// in shared memory)
constexpr int MAX_NMR = 256;

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R re, R im) {
  cx<R> z;
  z.re = re;
  z.im = im;
  return z;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return mk(a.re, -a.im); }
// i * a and -i * a
template <typename R>
__device__ __forceinline__ cx<R> times_i(cx<R> a) { return mk(-a.im, a.re); }
template <typename R>
__device__ __forceinline__ cx<R> times_mi(cx<R> a) { return mk(a.im, -a.re); }
// acc += a * b, acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cmac(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <typename R>
__device__ __forceinline__ void cmac_conj(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ---------------------------------------------------------------------------
// spinors: 4 spins x 3 colours, contiguous, vector loads and stores
// ---------------------------------------------------------------------------
template <typename R>
struct Spinor {
  cx<R> c[4][3];
};

// An FP32 spinor is 96 bytes at a multiple of 96 bytes from a 256-byte aligned
// block, so it is 32-byte aligned: three 256-bit loads (stores) move it, and a
// warp's load of (site, rhs) spinors uses every 32-byte sector it touches
// (16-byte loads at a 96-byte stride fetch each sector twice).
__device__ __forceinline__ void load_spinor(const cx<float>* p, Spinor<float>& s) {
  float* d = &s.c[0][0].re;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(d[8 * k]), "=f"(d[8 * k + 1]), "=f"(d[8 * k + 2]), "=f"(d[8 * k + 3]), "=f"(d[8 * k + 4]),
                   "=f"(d[8 * k + 5]), "=f"(d[8 * k + 6]), "=f"(d[8 * k + 7])
                 : "l"(reinterpret_cast<const float*>(p) + 8 * k));
}
__device__ __forceinline__ void load_spinor(const cx<double>* p, Spinor<double>& s) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const double2 v = __ldg(q + k);
    (&s.c[0][0])[k] = mk(v.x, v.y);
  }
}
__device__ __forceinline__ void store_spinor(cx<float>* p, const Spinor<float>& s) {
  const float* d = &s.c[0][0].re;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(reinterpret_cast<float*>(p) + 8 * k),
                 "f"(d[8 * k]), "f"(d[8 * k + 1]), "f"(d[8 * k + 2]), "f"(d[8 * k + 3]), "f"(d[8 * k + 4]),
                 "f"(d[8 * k + 5]), "f"(d[8 * k + 6]), "f"(d[8 * k + 7])
                 : "memory");
}
__device__ __forceinline__ void store_spinor(cx<double>* p, const Spinor<double>& s) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int k = 0; k < 12; ++k) q[k] = make_double2((&s.c[0][0])[k].re, (&s.c[0][0])[k].im);
}

// FP16 storage of a spinor (the FP16-storage operator and the preconditioner's
// FP16 blocks): 12 __half2 (re, im) q times one FP32 scale s, the largest |re|
// or |im| of the spinor, so every stored half lies in [-1, 1].
__device__ __forceinline__ void load_spinor_h(const __half2* __restrict__ q, float s, Spinor<float>& v) {
  const uint4* p = reinterpret_cast<const uint4*>(q);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 w = __ldg(p + k);
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __half2 h;
      memcpy(&h, &u[e], 4);
      const float2 f = __half22float2(h);
      (&v.c[0][0])[4 * k + e] = mk(f.x * s, f.y * s);
    }
  }
}

// rounds v into (q, s): s = max |re|, |im|; q = v / s to nearest FP16
__device__ __forceinline__ void store_spinor_h(__half2* __restrict__ q, float* __restrict__ s,
                                               const Spinor<float>& v) {
  float m = 0.0f;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const cx<float> c = (&v.c[0][0])[k];
    m = fmaxf(m, fmaxf(fabsf(c.re), fabsf(c.im)));
  }
  uint32_t u[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const cx<float> c = (&v.c[0][0])[k];
    const __half2 h = m > 0.0f ? __floats2half2_rn(c.re / m, c.im / m) : __floats2half2_rn(0.0f, 0.0f);
    memcpy(&u[k], &h, 4);
  }
  uint4* p = reinterpret_cast<uint4*>(q);
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
  *s = m;
}

template <typename R>
__device__ __forceinline__ void zero(Spinor<R>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) (&s.c[0][0])[k] = mk<R>(0, 0);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) completing on an mbarrier.
// Every wait is bounded: after MBAR_SPIN_LIMIT polls the caller gives up and
// reports an error instead of hanging.
// ---------------------------------------------------------------------------
constexpr int MBAR_SPIN_LIMIT = 1 << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// true when the phase completed, false when the wait gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int limit = MBAR_SPIN_LIMIT) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
// global -> shared bulk copy of `bytes` (multiple of 16, 16-byte aligned ends)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// 3x3 link matrices
// ---------------------------------------------------------------------------
template <typename R>
struct Link {
  cx<R> m[3][3];
};

__device__ __forceinline__ void load_link(const cx<float>* p, Link<float>& u) {
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 v = __ldg(q + k);
    (&u.m[0][0])[k] = mk(v.x, v.y);
  }
}
// The third row of an SU(3) link from its first two: the complex conjugate of
// their cross product (unitarity with det = 1).
__device__ __forceinline__ void complete_third_row(Link<float>& u) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    const cx<float> t = u.m[0][j1] * u.m[1][j2] - u.m[0][j2] * u.m[1][j1];
    u.m[2][j] = conjg(t);
  }
}
// An SU(3) link stored as its first two rows (6 complex numbers, 48 bytes,
// 16-byte aligned): three 16-byte loads instead of nine 8-byte ones.
__device__ __forceinline__ void load_link12(const cx<float>* p, Link<float>& u) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
  u.m[0][0] = mk(a.x, a.y);
  u.m[0][1] = mk(a.z, a.w);
  u.m[0][2] = mk(b.x, b.y);
  u.m[1][0] = mk(b.z, b.w);
  u.m[1][1] = mk(c.x, c.y);
  u.m[1][2] = mk(c.z, c.w);
  complete_third_row(u);
}
__device__ __forceinline__ void load_link(const cx<double>* p, Link<double>& u) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = __ldg(q + k);
    (&u.m[0][0])[k] = mk(v.x, v.y);
  }
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
// Division by a fixed divisor with a multiply-high and a shift (round-up magic
// number, exact for every dividend below 2^31).
struct FastDiv {
  uint32_t d = 1, m = 1;
  int l = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t div) : d(div) {
    l = 0;
    while ((1ull << l) < d) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// Site indices are 32-bit (the library limits the volume to 2^27 sites);
// element offsets are formed in 64-bit at the end.
struct Geom {
  int d[4];      // lattice extents
  int blk[4];    // SAP domain extents
  int nb[4];     // domains per direction
  int V;         // sites
  int Vd;        // sites per domain
  int nd;        // domains
  int su3;       // every link is unitary with det 1 (third rows may be rebuilt)
  FastDiv fd0, fd1, fd2;      // lattice extents x, y, z
  FastDiv fb0, fb1, fb2;      // domain extents x, y, z
  FastDiv fVd, fhalf, fnb1, fnb2;  // sites per domain, nb[0]/2, nb[1], nb[2]
};

inline void geom_init_divisors(Geom& g) {
  g.fd0 = FastDiv(g.d[0]);
  g.fd1 = FastDiv(g.d[1]);
  g.fd2 = FastDiv(g.d[2]);
  g.fb0 = FastDiv(g.blk[0]);
  g.fb1 = FastDiv(g.blk[1]);
  g.fb2 = FastDiv(g.blk[2]);
  g.fVd = FastDiv(g.Vd);
  g.fhalf = FastDiv(g.nb[0] / 2 > 0 ? g.nb[0] / 2 : 1);
  g.fnb1 = FastDiv(g.nb[1]);
  g.fnb2 = FastDiv(g.nb[2]);
}

__device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
  const uint32_t q1 = g.fd0.div(s);
  c[0] = s - q1 * g.d[0];
  const uint32_t q2 = g.fd1.div(q1);
  c[1] = q1 - q2 * g.d[1];
  const uint32_t q3 = g.fd2.div(q2);
  c[2] = q2 - q3 * g.d[2];
  c[3] = q3;
}
__device__ __forceinline__ int site_index(const Geom& g, const int c[4]) {
  return c[0] + g.d[0] * (c[1] + g.d[1] * (c[2] + g.d[2] * c[3]));
}

// The k-th domain of colour `colour` (colour = parity of the sum of the domain
// coordinates), with domains enumerated lexicographically inside each colour.
// Rows of domains along x hold nb[0]/2 domains of each colour because nb[0]
// is even.
__device__ __forceinline__ void colour_domain(const Geom& g, int colour, int k, int b[4]) {
  const int half = g.nb[0] >> 1;
  const int row0 = g.fhalf.div(k);
  const int j = 2 * (k - row0 * half);
  const int row1 = g.fnb1.div(row0);
  b[1] = row0 - row1 * g.nb[1];
  const int row2 = g.fnb2.div(row1);
  b[2] = row1 - row2 * g.nb[2];
  b[3] = row2;
  const int p = (b[1] + b[2] + b[3]) & 1;
  b[0] = j + (colour ^ p);
}

// Site coordinates of slot `slot` of colour `colour`: slot = k * Vd + local,
// local lexicographic inside the domain.  Also returns the local coordinates.
__device__ __forceinline__ void colour_slot_coords(const Geom& g, int colour, int slot, int c[4], int lc[4],
                                                   int* kdom) {
  const int k = g.fVd.div(slot);
  int l = slot - k * g.Vd;
  int b[4];
  colour_domain(g, colour, k, b);
  int q = g.fb0.div(l);
  lc[0] = l - q * g.blk[0];
  l = q;
  q = g.fb1.div(l);
  lc[1] = l - q * g.blk[1];
  l = q;
  q = g.fb2.div(l);
  lc[2] = l - q * g.blk[2];
  lc[3] = q;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) c[mu] = b[mu] * g.blk[mu] + lc[mu];
  *kdom = k;
}

// ---------------------------------------------------------------------------
// Spin projection of the Wilson hopping term in the chiral basis.
// (1 -/+ gamma_mu) psi = (h0, h1, lower(h0, h1)): project to the two upper
// spin components h, multiply h by the link, and rebuild the lower two.
// SIGN = -1 selects (1 - gamma_mu) (forward hop), +1 (1 + gamma_mu) (backward).
// ---------------------------------------------------------------------------
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void project(const Spinor<R>& p, cx<R> h[2][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (MU == 0) {  // gamma_1: pairs (0,3), (1,2) with factor -/+ i
      if (SIGN < 0) { h[0][a] = p.c[0][a] + times_i(p.c[3][a]); h[1][a] = p.c[1][a] + times_i(p.c[2][a]); }
      else          { h[0][a] = p.c[0][a] + times_mi(p.c[3][a]); h[1][a] = p.c[1][a] + times_mi(p.c[2][a]); }
    } else if (MU == 1) {  // gamma_2
      if (SIGN < 0) { h[0][a] = p.c[0][a] + p.c[3][a]; h[1][a] = p.c[1][a] - p.c[2][a]; }
      else          { h[0][a] = p.c[0][a] - p.c[3][a]; h[1][a] = p.c[1][a] + p.c[2][a]; }
    } else if (MU == 2) {  // gamma_3
      if (SIGN < 0) { h[0][a] = p.c[0][a] + times_i(p.c[2][a]); h[1][a] = p.c[1][a] + times_mi(p.c[3][a]); }
      else          { h[0][a] = p.c[0][a] + times_mi(p.c[2][a]); h[1][a] = p.c[1][a] + times_i(p.c[3][a]); }
    } else {  // gamma_4
      if (SIGN < 0) { h[0][a] = p.c[0][a] - p.c[2][a]; h[1][a] = p.c[1][a] - p.c[3][a]; }
      else          { h[0][a] = p.c[0][a] + p.c[2][a]; h[1][a] = p.c[1][a] + p.c[3][a]; }
    }
  }
}

// acc += (1 -/+ gamma_mu) rebuilt from the colour-rotated half spinor w
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void reconstruct_add(Spinor<R>& acc, const cx<R> w[2][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc.c[0][a] = acc.c[0][a] + w[0][a];
    acc.c[1][a] = acc.c[1][a] + w[1][a];
    if (MU == 0) {
      if (SIGN < 0) { acc.c[2][a] = acc.c[2][a] + times_mi(w[1][a]); acc.c[3][a] = acc.c[3][a] + times_mi(w[0][a]); }
      else          { acc.c[2][a] = acc.c[2][a] + times_i(w[1][a]);  acc.c[3][a] = acc.c[3][a] + times_i(w[0][a]); }
    } else if (MU == 1) {
      if (SIGN < 0) { acc.c[2][a] = acc.c[2][a] - w[1][a]; acc.c[3][a] = acc.c[3][a] + w[0][a]; }
      else          { acc.c[2][a] = acc.c[2][a] + w[1][a]; acc.c[3][a] = acc.c[3][a] - w[0][a]; }
    } else if (MU == 2) {
      if (SIGN < 0) { acc.c[2][a] = acc.c[2][a] + times_mi(w[0][a]); acc.c[3][a] = acc.c[3][a] + times_i(w[1][a]); }
      else          { acc.c[2][a] = acc.c[2][a] + times_i(w[0][a]);  acc.c[3][a] = acc.c[3][a] + times_mi(w[1][a]); }
    } else {
      if (SIGN < 0) { acc.c[2][a] = acc.c[2][a] - w[0][a]; acc.c[3][a] = acc.c[3][a] - w[1][a]; }
      else          { acc.c[2][a] = acc.c[2][a] + w[0][a]; acc.c[3][a] = acc.c[3][a] + w[1][a]; }
    }
  }
}

// w = U h (forward) or U^dagger h (backward), times the boundary phase
template <bool DAGGER, typename R>
__device__ __forceinline__ void link_times(const Link<R>& u, const cx<R> h[2][3], R phase, cx<R> w[2][3]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (DAGGER) cmac_conj(acc, u.m[b][a], h[sp][b]);
        else cmac(acc, u.m[a][b], h[sp][b]);
      }
      w[sp][a] = phase * acc;
    }
}

// ---------------------------------------------------------------------------
// Site-local Hermitian spin-colour matrices that are block diagonal in
// chirality (the clover term and its inverse: sigma_{mu nu} commutes with
// gamma_5 = diag(1, 1, -1, -1) in the chiral basis).  Per site two 6 x 6
// blocks, spins 0-1 and spins 2-3, index 3 * spin + colour inside a block;
// each block packed as its 6 real diagonal entries, then the 15 entries above
// the diagonal row by row as (re, im): 36 reals per block, 72 per site.
// ---------------------------------------------------------------------------
constexpr int HERM_PER_SITE = 72;

__host__ __device__ constexpr int herm_off(int i, int j) {  // i < j
  return 6 + 2 * (i * 6 - i * (i + 1) / 2 + (j - i - 1));
}

// y = M x for the packed matrix M of one site (m: its 72 reals); each entry is
// loaded where it is used (the off-diagonal ones twice, from L1), which keeps
// few registers live inside kernels that are already near their limit
template <typename R>
__device__ __forceinline__ void herm_apply(const R* __restrict__ m, const Spinor<R>& x, Spinor<R>& y) {
  const cx<R>* xv = &x.c[0][0];
  cx<R>* yv = &y.c[0][0];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const R* mb = m + 36 * b;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const R d = __ldg(mb + i);
      const cx<R> xi = xv[6 * b + i];
      cx<R> acc = mk(d * xi.re, d * xi.im);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j == i) continue;
        const int o = i < j ? herm_off(i, j) : herm_off(j, i);
        const R re = __ldg(mb + o), im = __ldg(mb + o + 1);
        cmac(acc, i < j ? mk(re, im) : mk(re, -im), xv[6 * b + j]);
      }
      yv[6 * b + i] = acc;
    }
  }
}

}  // namespace mbicg
