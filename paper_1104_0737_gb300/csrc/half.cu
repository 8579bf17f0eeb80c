// half.cu — FP16 storage of spinor blocks and links, FP32 arithmetic.
//
// Storage format (the internal site-major order of the FP32 blocks):
//   spinors  q[site][rhs][12] __half2 (re, im), 48 bytes, with one FP32 scale
//            s[site][rhs] = the largest |re| or |im| of that spinor; the value
//            represented is q * s, so every stored half lies in [-1, 1];
//   links    the first two rows of each link, [site][mu][6] __half2 (24 bytes),
//            no scale (|U_ab| <= 1 for SU(3)); the third row is rebuilt in FP32
//            as the conjugate cross product of the first two.
// The operator (Sec. 2.1, the hopping term of the Wilson-Dirac matrix) reads
// FP16 neighbours and links, accumulates in FP32 and rounds its result into the
// same format.  Per site and column it moves L x (2 x 52) + 96 bytes instead of
// L x 192 + 192 in FP32 with two-row links.
#include <cuda_fp16.h>

#include "internal.h"

namespace mbicg {

namespace {

constexpr int HT = 256;

__device__ __forceinline__ void load_link_h(const __half2* __restrict__ l, Link<float>& u) {
  const uint2* p = reinterpret_cast<const uint2*>(l);
  float2 f[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint2 w = __ldg(p + k);
    __half2 a, b;
    memcpy(&a, &w.x, 4);
    memcpy(&b, &w.y, 4);
    f[2 * k] = __half22float2(a);
    f[2 * k + 1] = __half22float2(b);
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) (&u.m[0][0])[e] = mk(f[e].x, f[e].y);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    const cx<float> t = u.m[0][j1] * u.m[1][j2] - u.m[0][j2] * u.m[1][j1];
    u.m[2][j] = conjg(t);
  }
}

template <int MU, int SIGN>
__device__ __forceinline__ void hop_h(Spinor<float>& acc, const __half2* __restrict__ q, const float* __restrict__ sc,
                                      const __half2* __restrict__ l16, int sn, int sl, int L, int rhs, bool flip) {
  Spinor<float> p;
  load_spinor_h(q + ((size_t)sn * L + rhs) * 12, __ldg(sc + (size_t)sn * L + rhs), p);
  Link<float> u;
  load_link_h(l16 + ((size_t)sl * 4 + MU) * 6, u);
  cx<float> h[2][3], w[2][3];
  project<MU, SIGN>(p, h);
  link_times<(SIGN > 0)>(u, h, flip ? -1.0f : 1.0f, w);
  reconstruct_add<MU, SIGN>(acc, w);
}

template <int MU>
__device__ __forceinline__ void hops_h(const Geom& g, Spinor<float>& acc, const __half2* __restrict__ q,
                                       const float* __restrict__ sc, const __half2* __restrict__ l16, int s,
                                       const int c[4], int stride, int L, int rhs) {
  const int dm = g.d[MU];
  {
    const bool wrap = c[MU] == dm - 1;
    const int sn = wrap ? s - (dm - 1) * stride : s + stride;
    hop_h<MU, -1>(acc, q, sc, l16, sn, s, L, rhs, MU == 3 && wrap);
  }
  {
    const bool wrap = c[MU] == 0;
    const int sn = wrap ? s + (dm - 1) * stride : s - stride;
    hop_h<MU, 1>(acc, q, sc, l16, sn, sn, L, rhs, MU == 3 && wrap);
  }
}

// one thread per (site, column): out = in - kappa * hops, FP16 in and out
__global__ void __launch_bounds__(384, 2) k_dslash_half(Geom g, const __half2* __restrict__ l16,
                                                        const __half2* __restrict__ q, const float* __restrict__ sc,
                                                        __half2* __restrict__ qo, float* __restrict__ so, int L,
                                                        float kappa) {
  const int rhs = threadIdx.x;
  const int s = blockIdx.x * blockDim.y + threadIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  Spinor<float> acc;
  zero(acc);
  const int st1 = g.d[0], st2 = st1 * g.d[1], st3 = st2 * g.d[2];
  hops_h<0>(g, acc, q, sc, l16, s, c, 1, L, rhs);
  hops_h<1>(g, acc, q, sc, l16, s, c, st1, L, rhs);
  hops_h<2>(g, acc, q, sc, l16, s, c, st2, L, rhs);
  hops_h<3>(g, acc, q, sc, l16, s, c, st3, L, rhs);
  Spinor<float> p;
  const size_t i = (size_t)s * L + rhs;
  load_spinor_h(q + i * 12, __ldg(sc + i), p);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    cx<float>& o = (&acc.c[0][0])[k];
    const cx<float> v = (&p.c[0][0])[k];
    o = mk(fmaf(-kappa, o.re, v.re), fmaf(-kappa, o.im, v.im));
  }
  store_spinor_h(qo + i * 12, so + i, acc);
}

// ABI FP64 [site][spin][colour][rhs] -> FP16 + scale, one thread per (site, rhs);
// the scale is the FP64 max-abs rounded to FP32, the quotient rounded once
// from FP64 to FP16
__global__ void k_abi_to_half(long long nsite, int L, const cx<double>* __restrict__ in, __half2* __restrict__ q,
                              float* __restrict__ sc) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsite * L) return;
  const long long site = idx / L;
  const int rhs = (int)(idx - site * L);
  cx<double> v[12];
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[k] = in[((size_t)site * 12 + k) * L + rhs];
    m = fmax(m, fmax(fabs(v[k].re), fabs(v[k].im)));
  }
  const float s = (float)m;
  const double ds = (double)s;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    __half2 h;
    h.x = s > 0.0f ? __double2half(v[k].re / ds) : __float2half(0.0f);
    h.y = s > 0.0f ? __double2half(v[k].im / ds) : __float2half(0.0f);
    q[idx * 12 + k] = h;
  }
  sc[idx] = s;
}

// FP16 + scale -> ABI FP64 (exact: an 11-bit by 24-bit product)
__global__ void k_half_to_abi(long long nsite, int L, const __half2* __restrict__ q, const float* __restrict__ sc,
                              cx<double>* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nsite * L) return;
  const long long site = idx / L;
  const int rhs = (int)(idx - site * L);
  const double s = (double)sc[idx];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 f = __half22float2(q[idx * 12 + k]);
    out[((size_t)site * 12 + k) * L + rhs] = mk((double)f.x * s, (double)f.y * s);
  }
}

// links: the first two rows of each FP64 link rounded to FP16
__global__ void k_links_to_half(long long nlinks, const cx<double>* __restrict__ in, __half2* __restrict__ l16) {
  for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks;
       l += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const cx<double> v = in[l * 9 + e];
      __half2 h;
      h.x = __double2half(v.re);
      h.y = __double2half(v.im);
      l16[l * 6 + e] = h;
    }
  }
}

// FP32 internal block <-> FP16 storage, one thread per spinor (the same
// [site][rhs] order, so the conversion is elementwise per spinor)
__global__ void k_block_to_half(long long n, const cx<float>* __restrict__ in, __half2* __restrict__ q,
                                float* __restrict__ sc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Spinor<float> v;
  load_spinor(in + i * 12, v);
  store_spinor_h(q + i * 12, sc + i, v);
}

__global__ void k_half_to_block(long long n, const __half2* __restrict__ q, const float* __restrict__ sc,
                                cx<float>* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Spinor<float> v;
  load_spinor_h(q + i * 12, __ldg(sc + i), v);
  store_spinor(out + i * 12, v);
}

unsigned grid_of(long long n) { return (unsigned)((n + HT - 1) / HT); }

}  // namespace

void abi_to_half(const Exec& ex, long long nsite, int L, const cx<double>* in, __half2* q, float* sc) {
  k_abi_to_half<<<grid_of(nsite * L), HT, 0, ex.stream>>>(nsite, L, in, q, sc);
  ++*ex.launches;
}

void block_to_half(const Exec& ex, long long nspinor, const cx<float>* in, __half2* q, float* sc) {
  k_block_to_half<<<grid_of(nspinor), HT, 0, ex.stream>>>(nspinor, in, q, sc);
  ++*ex.launches;
}

void half_to_block(const Exec& ex, long long nspinor, const __half2* q, const float* sc, cx<float>* out) {
  k_half_to_block<<<grid_of(nspinor), HT, 0, ex.stream>>>(nspinor, q, sc, out);
  ++*ex.launches;
}

void half_to_abi(const Exec& ex, long long nsite, int L, const __half2* q, const float* sc, cx<double>* out) {
  k_half_to_abi<<<grid_of(nsite * L), HT, 0, ex.stream>>>(nsite, L, q, sc, out);
  ++*ex.launches;
}

void links_to_half(const Exec& ex, long long nsite, const cx<double>* in, __half2* l16) {
  const long long n = nsite * 4;
  k_links_to_half<<<(unsigned)std::min<long long>(grid_of(n), 8 * 152), HT, 0, ex.stream>>>(n, in, l16);
  ++*ex.launches;
}

void dslash_half(const Exec& ex, const Geom& g, const __half2* l16, const __half2* q, const float* sc, __half2* qo,
                 float* so, int L, double kappa) {
  int S = 1;
  while (S * 2 * L <= 384) S *= 2;
  const dim3 block(L, S);
  const int grid = (g.V + S - 1) / S;
  k_dslash_half<<<(unsigned)grid, block, 0, ex.stream>>>(g, l16, q, sc, qo, so, L, (float)kappa);
  ++*ex.launches;
}

}  // namespace mbicg
