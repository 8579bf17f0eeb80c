"""FP16 storage of the operator (Sec. 2.1 hopping term; FP16 blocks with one
scale per (site, rhs), FP16 link rows, FP32 arithmetic) through the C ABI
(mbicg_apply_D with MBICG_FP16), against the oracle's FP16 storage format."""
import numpy as np
import pytest

import oracle
import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def comps(a):
    """(V, 4, 3, L) complex -> (V, L, 24) reals of each (site, rhs) spinor."""
    V, L = a.shape[0], a.shape[-1]
    return np.stack([a.real, a.imag], -1).reshape(V, 12, L, 2).transpose(0, 2, 1, 3).reshape(V, L, 24)


@pytest.mark.parametrize("dims,L", [((8, 8, 8, 16), 12), ((6, 4, 2, 10), 5), ((4, 4, 4, 4), 1)])
def test_fp16_storage_round_trip_is_the_oracle_format(dims, L):
    """kappa = 0: the operator is the identity, so the result is the input as
    FP16 storage represents it, bit for bit."""
    ctx, U = make_ctx(dims, 0.5, seed=61)
    try:
        psi = synth.gaussian_source(dims, L, seed=62)
        psi[3] = 0  # a zero spinor keeps scale 0
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, 0.0, mb.MBICG_FP16)
        assert np.array_equal(out, oracle.quantize_fp16(psi))
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.parametrize("dims,L", [((8, 8, 8, 16), 12), ((6, 4, 2, 10), 5), ((4, 4, 4, 4), 3)])
def test_fp16_operator_matches_oracle_on_fp16_inputs(oracle_mod, dims, L):
    """The oracle applied to the FP16-represented links and input, rounded into
    the FP16 format: equal up to one FP16 step of the output scale where the
    FP32 and FP64 sums fall on either side of a rounding boundary."""
    ctx, U = make_ctx(dims, 0.5, seed=63)
    try:
        psi = synth.gaussian_source(dims, L, seed=64)
        kappa = 0.13
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP16)
        exp = oracle.quantize_fp16(oracle_mod.apply_D(dims, oracle.quantize_links_fp16(U), kappa,
                                                      oracle.quantize_fp16(psi)))
        g, e = comps(out), comps(exp)
        s = np.abs(e).max(axis=2, keepdims=True)
        assert np.all(np.abs(g - e) <= 2.0 ** -10 * s)
        # the two scales may differ in their last FP32 bit (FP32 vs FP64
        # max-abs), which moves every component by ~2^-24 s; FP16 rounding
        # flips are larger and rare
        assert np.mean(np.abs(g - e) > 2.0 ** -20 * s) < 0.05
    finally:
        mb.mbicg_destroy(ctx)


def test_fp16_operator_error_against_fp64_is_within_its_bound(oracle_mod):
    """Against the FP64 operator on the unrounded data: per component at most
    2^-12 (s_x + s_out + 42 kappa sum_n s_n) + FP32 arithmetic, where s is the
    max-abs scale of a spinor and n runs over the 8 neighbours (each hop term
    has 6 products of a link entry (|U_ab| <= 1, rounded by <= 2^-12 per part
    in rows 0-1, <= 6 2^-12 in the rebuilt row 2) with an input component
    (rounded by <= 2^-12 s_n)).  Also records the typical error."""
    dims, L = (8, 8, 8, 16), 12
    ctx, U = make_ctx(dims, 0.5, seed=65)
    try:
        psi = synth.gaussian_source(dims, L, seed=66)
        kappa = 0.13
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP16)
        ref = oracle_mod.apply_D(dims, U, kappa, psi)
        g, r, p = comps(out), comps(ref), comps(psi)
        s_in = np.abs(p).max(axis=2)                      # (V, L)
        s_out = np.abs(r).max(axis=2)
        # neighbour scales: sum over the 8 neighbours of each site
        V = psi.shape[0]
        x = np.arange(V)
        c = np.stack([x % dims[0], (x // dims[0]) % dims[1], (x // (dims[0] * dims[1])) % dims[2],
                      x // (dims[0] * dims[1] * dims[2])], 1)
        nsum = np.zeros_like(s_in)
        for mu in range(4):
            for d in (1, -1):
                cn = c.copy()
                cn[:, mu] = (cn[:, mu] + d) % dims[mu]
                sn = cn[:, 0] + dims[0] * (cn[:, 1] + dims[1] * (cn[:, 2] + dims[2] * cn[:, 3]))
                nsum += s_in[sn]
        bound = 2.0 ** -12 * (s_in + s_out + 42 * kappa * nsum) + 1e-6 * (s_in + nsum)
        err = np.abs(g - r).max(axis=2)
        assert np.all(err <= bound)
        rel = np.linalg.norm(g - r, axis=2) / np.linalg.norm(r, axis=2)
        assert np.median(rel) < 1e-3 and np.max(rel) < 1e-2, (np.median(rel), np.max(rel))
    finally:
        mb.mbicg_destroy(ctx)


def test_fp16_needs_su3_links():
    dims = (4, 4, 4, 4)
    ctx = mb.mbicg_create(dims)
    try:
        mb.mbicg_load_gauge(ctx, 1.05 * synth.su3_links(dims, 0.5, 67))
        psi = synth.gaussian_source(dims, 2, seed=68)
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_apply_D(ctx, psi, np.empty_like(psi), 2, 0.1, mb.MBICG_FP16)
        assert e.value.status == mb.MBICG_EINVAL
    finally:
        mb.mbicg_destroy(ctx)
