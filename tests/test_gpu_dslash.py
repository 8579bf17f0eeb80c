"""Parity of the CUDA block Wilson-Dirac operator (Sec. 2.1) with the FP64
oracle, through the C ABI: 1e-13 relative per-site norm in FP64, 1e-6 in FP32.
Lattices are chosen so the CTAs of S sites leave a ragged tail, with L from 1
to the maximum 16."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx, rel_site_norm

pytestmark = pytest.mark.gpu

CASES = [((4, 4, 4, 4), 4), ((6, 2, 4, 10), 12), ((8, 8, 8, 16), 1), ((2, 2, 2, 2), 16),
         ((4, 6, 2, 10), 3), ((10, 6, 6, 4), 7),
         # L = 4, 8, 12 on lattices with extents 32 and 2 (every hop of a
         # site wraps in y, z and t at once on the last one)
         ((8, 8, 8, 16), 12), ((16, 8, 4, 4), 8), ((32, 2, 2, 4), 12), ((8, 4, 2, 2), 4)]


@pytest.mark.parametrize("dims,L", CASES)
def test_dslash_fp64_and_fp32_match_oracle(oracle_mod, dims, L):
    ctx, U = make_ctx(dims, 0.5, seed=11)
    try:
        psi = synth.gaussian_source(dims, L, seed=12)
        kappa = 0.1375
        ref = oracle_mod.apply_D(dims, U, kappa, psi)
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP64)
        assert rel_site_norm(out, ref) < 1e-13
        mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP32)
        assert rel_site_norm(out, ref) < 1e-6
    finally:
        mb.mbicg_destroy(ctx)


def test_dslash_device_pointers_and_stream():
    torch = pytest.importorskip("torch")
    dims, L = (8, 4, 4, 8), 5
    ctx, U = make_ctx(dims, 0.5, seed=21)
    try:
        psi = synth.gaussian_source(dims, L, seed=22)
        host = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, host, L, 0.12, mb.MBICG_FP64)
        d_in = torch.from_numpy(psi).cuda()
        d_out = torch.empty_like(d_in)
        mb.mbicg_apply_D(ctx, d_in, d_out, L, 0.12, mb.MBICG_FP64)
        torch.cuda.synchronize()
        # same kernels, same inputs: bitwise identical
        assert np.array_equal(d_out.cpu().numpy(), host)
    finally:
        mb.mbicg_destroy(ctx)


def test_dslash_is_deterministic_and_columnwise():
    dims = (4, 4, 4, 8)
    ctx, U = make_ctx(dims, 0.5, seed=31)
    try:
        B = synth.gaussian_source(dims, 6, seed=32)
        a = np.empty_like(B)
        b = np.empty_like(B)
        mb.mbicg_apply_D(ctx, B, a, 6, 0.13, mb.MBICG_FP32)
        mb.mbicg_apply_D(ctx, B, b, 6, 0.13, mb.MBICG_FP32)
        assert np.array_equal(a, b)
        one = np.empty_like(B[..., 2:3])
        mb.mbicg_apply_D(ctx, np.ascontiguousarray(B[..., 2:3]), one, 1, 0.13, mb.MBICG_FP32)
        assert np.array_equal(one[..., 0], a[..., 2])
    finally:
        mb.mbicg_destroy(ctx)


def test_dslash_errors():
    dims = (4, 4, 4, 4)
    ctx = mb.mbicg_create(dims)
    try:
        psi = synth.gaussian_source(dims, 2, seed=1)
        out = np.empty_like(psi)
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_apply_D(ctx, psi, out, 2, 0.1, mb.MBICG_FP64)
        assert e.value.status == mb.MBICG_ENOGAUGE
        U = synth.su3_links(dims, 0.5, seed=2)
        U[3, 1, 0, 0] = np.nan
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_load_gauge(ctx, U)
        assert e.value.status == mb.MBICG_ENAN
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_apply_D(ctx, psi, out, 2, 0.1, mb.MBICG_FP64)
        assert e.value.status == mb.MBICG_ENOGAUGE  # a failed load leaves no field
        mb.mbicg_load_gauge(ctx, synth.su3_links(dims, 0.5, seed=2))
        for L in (0, 17):
            with pytest.raises(mb.MbicgError) as e:
                mb.mbicg_apply_D(ctx, psi, out, L, 0.1, mb.MBICG_FP64)
            assert e.value.status == mb.MBICG_EINVAL
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_apply_D(ctx, psi, out, 2, 0.1, 7)  # no such precision
        assert e.value.status == mb.MBICG_EINVAL
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.slow
def test_dslash_full_size_32c64_L12(oracle_mod):
    """The benchmark's lattice and launch configuration (32^3 x 64, L = 12,
    FP32) against the oracle on every site."""
    dims, L = (32, 32, 32, 64), 12
    ctx, U = make_ctx(dims, 0.5, seed=1003)
    try:
        psi = synth.gaussian_source(dims, L, seed=2003)
        kappa = 0.14
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP32)
        ref = oracle_mod.apply_D(dims, U, kappa, psi)
        assert rel_site_norm(out, ref) < 1e-6
    finally:
        mb.mbicg_destroy(ctx)


def test_dslash_fp32_on_links_that_are_not_su3(oracle_mod):
    """The FP32 operator uses all nine link entries, so a field that is not
    SU(3) (links scaled by 1.05) matches the oracle as well as an SU(3) one,
    for L = 12 and for the first four columns alone."""
    dims, L = (8, 8, 8, 16), 12
    psi = synth.gaussian_source(dims, L, seed=52)
    kappa = 0.13
    for scale in (1.0, 1.05):
        U = scale * synth.su3_links(dims, 0.5, 51)
        ctx = mb.mbicg_create(dims)
        try:
            mb.mbicg_load_gauge(ctx, U)
            ref = oracle_mod.apply_D(dims, U, kappa, psi)
            out = np.empty_like(psi)
            mb.mbicg_apply_D(ctx, psi, out, L, kappa, mb.MBICG_FP32)
            assert rel_site_norm(out, ref) < 1e-6, scale
            # columns 0..3 alone
            part = np.ascontiguousarray(psi[..., :4])
            out4 = np.empty_like(part)
            mb.mbicg_apply_D(ctx, part, out4, 4, kappa, mb.MBICG_FP32)
            assert rel_site_norm(out4, np.ascontiguousarray(ref[..., :4])) < 1e-6, scale
        finally:
            mb.mbicg_destroy(ctx)
