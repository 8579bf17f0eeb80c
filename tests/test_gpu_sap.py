"""Parity of the CUDA SAP preconditioner (Sec. 2.2) with the FP64 oracle
through the C ABI, for per-column and block-shared MR step lengths, in FP64
(1e-12 relative per-site norm) and FP32 (1e-5)."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx, rel_site_norm

pytestmark = pytest.mark.gpu

CASES = [
    # dims, block, L, ncycle, nmr, kappa
    ((4, 4, 4, 4), (2, 2, 2, 2), 4, 4, 4, 0.12),     # the plain FP64 4^4 configuration
    ((8, 8, 8, 16), (4, 4, 4, 4), 12, 4, 4, 0.125),  # 8^3 x 16, 4^4 domains
    ((8, 4, 4, 8), (2, 2, 2, 4), 3, 2, 5, 0.13),     # anisotropic domains
    ((4, 4, 4, 8), (1, 1, 1, 1), 2, 1, 1, 0.13),     # single-site domains
    ((16, 16, 16, 16), (8, 8, 8, 8), 2, 2, 3, 0.146),  # 8^4 domains (the benchmark's shape)
]


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,kappa", CASES)
@pytest.mark.parametrize("mr_mode", [mb.MBICG_MR_COLUMN, mb.MBICG_MR_BLOCK])
@pytest.mark.parametrize("fused", ["1", "0"])
def test_sap_matches_oracle(oracle_mod, monkeypatch, dims, block, L, ncycle, nmr, kappa, mr_mode,
                            fused):
    """fused = 1: FP32 sweeps of 8^4 and 4^4 domains run the on-chip cluster
    kernel; fused = 0 forces the multi-kernel path everywhere."""
    monkeypatch.setenv("MBICG_SAP_FUSED", fused)
    ctx, U = make_ctx(dims, 0.5, seed=41)
    try:
        eta = synth.gaussian_source(dims, L, seed=42)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=mr_mode)
        out = np.empty_like(eta)
        for prec, tol in ((mb.MBICG_FP64, 1e-12), (mb.MBICG_FP32, 1e-5)):
            p = mb.mbicg_default_params(ncycle=ncycle, nmr=nmr, block=block, mr_mode=mr_mode,
                                        prec_sap=prec)
            mb.mbicg_sap_precond(ctx, eta, out, L, kappa, p)
            assert rel_site_norm(out, ref) < tol, prec
    finally:
        mb.mbicg_destroy(ctx)


def test_sap_rejects_bad_blocking_and_modes():
    dims = (8, 8, 8, 8)
    ctx, _ = make_ctx(dims, 0.5, seed=1)
    try:
        eta = synth.gaussian_source(dims, 1, seed=2)
        out = np.empty_like(eta)
        for blk in [(8, 4, 4, 4), (3, 4, 4, 4), (2, 2, 2, 0)]:  # 1 domain in x; 3 does not divide 8
            p = mb.mbicg_default_params(block=blk)
            with pytest.raises(mb.MbicgError) as e:
                mb.mbicg_sap_precond(ctx, eta, out, 1, 0.12, p)
            assert e.value.status == mb.MBICG_EINVAL
        p = mb.mbicg_default_params(block=(4, 4, 4, 4), mr_mode=mb.MBICG_MR_FROZEN)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_sap_precond(ctx, eta, out, 1, 0.12, p)
        ctx2 = mb.mbicg_create((12, 8, 8, 8))
        mb.mbicg_load_gauge(ctx2, synth.su3_links((12, 8, 8, 8), 0.5, 3))
        e2 = synth.gaussian_source((12, 8, 8, 8), 1, seed=4)
        with pytest.raises(mb.MbicgError):  # 3 domains in x: no checkerboard
            mb.mbicg_sap_precond(ctx2, e2, np.empty_like(e2), 1, 0.12,
                                 mb.mbicg_default_params(block=(4, 4, 4, 4)))
        mb.mbicg_destroy(ctx2)
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.parametrize("dims,block", [((16, 16, 16, 16), (8, 8, 8, 8)), ((8, 8, 8, 16), (4, 4, 4, 4))])
def test_sap_non_su3_links(oracle_mod, monkeypatch, dims, block):
    """The on-chip sweep keeps two rows of each link and rebuilds the third
    from unitarity; a gauge field that is not SU(3) (links scaled by 1.05)
    must still give the oracle's result, by the multi-kernel path."""
    monkeypatch.setenv("MBICG_SAP_FUSED", "1")
    U = 1.05 * synth.su3_links(dims, 0.5, 77)
    ctx = mb.mbicg_create(dims)
    try:
        mb.mbicg_load_gauge(ctx, U)
        eta = synth.gaussian_source(dims, 3, seed=78)
        ref = oracle_mod.sap(dims, block, U, 0.12, 2, 3, eta, mr_mode=mb.MBICG_MR_COLUMN)
        out = np.empty_like(eta)
        p = mb.mbicg_default_params(ncycle=2, nmr=3, block=block, mr_mode=mb.MBICG_MR_COLUMN,
                                    prec_sap=mb.MBICG_FP32)
        mb.mbicg_sap_precond(ctx, eta, out, 3, 0.12, p)
        assert rel_site_norm(out, ref) < 1e-5
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.slow
def test_sap_full_size_32c64_L12(oracle_mod):
    """The benchmark's lattice, domains and launch configuration of the fused
    sweep (32^3 x 64, 8^4 domains split over 8-CTA clusters, L = 12, FP32),
    with per-column MR step lengths (the mode the oracle reproduces without
    the solver's recorded table), one cycle of two MR steps to keep the oracle
    within a minute: every site against the oracle."""
    dims, block, L = (32, 32, 32, 64), (8, 8, 8, 8), 12
    ctx, U = make_ctx(dims, 0.5, seed=1003)
    try:
        eta = synth.gaussian_source(dims, L, seed=2003)
        ref = oracle_mod.sap(dims, block, U, 0.14774, 1, 2, eta, mr_mode=mb.MBICG_MR_COLUMN)
        out = np.empty_like(eta)
        p = mb.mbicg_default_params(ncycle=1, nmr=2, block=block, mr_mode=mb.MBICG_MR_COLUMN,
                                    prec_sap=mb.MBICG_FP32)
        mb.mbicg_sap_precond(ctx, eta, out, L, 0.14774, p)
        assert rel_site_norm(out, ref) < 1e-5
    finally:
        mb.mbicg_destroy(ctx)
