"""The SAP preconditioner (Sec. 2.2) with its blocks in FP16 storage
(prec_sap = MBICG_FP16: input, output, colour residual and psi held in HBM as
FP16 spinors times one FP32 scale per (site, column); FP32 arithmetic, FP32
links, the MR state on chip in FP32) against the FP64 oracle.

Tolerance.  Rounding a spinor into the format changes each component by at
most 2^-11 (FP16's unit roundoff) of the spinor's largest component.  One
application of M rounds its input once and, per colour sweep, the residual
and psi once each: 2 + 4 ncycle roundings, each carried on by operators of
norm O(1) (the domain solves, the residual update).  The test asserts
(2 + 4 ncycle) 2^-11 for the relative error of the whole block (5e-3 at
ncycle = 2) and 2e-2 per site (a site's error is relative to its own scale,
and its value can be smaller than what its neighbours contribute to it)."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

U_HALF = 2.0 ** -11


def errors(out, ref):
    V = ref.shape[0]
    d = np.linalg.norm((out - ref).reshape(V, -1), axis=1)
    r = np.linalg.norm(ref.reshape(V, -1), axis=1)
    return float(np.linalg.norm(out - ref) / np.linalg.norm(ref)), float(np.max(d / r))


CASES = [
    # dims, block, L, ncycle, nmr, kappa
    ((16, 16, 16, 16), (8, 8, 8, 8), 12, 2, 4, 0.146),   # 8-CTA cluster sweep
    ((8, 8, 8, 16), (4, 4, 4, 4), 12, 2, 4, 0.125),      # one-CTA sweep
    ((8, 8, 8, 16), (4, 4, 4, 4), 3, 1, 3, 0.13),
]


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,kappa", CASES)
def test_fp16_sap_per_column_matches_oracle(oracle_mod, dims, block, L, ncycle, nmr, kappa):
    ctx, U = make_ctx(dims, 0.5, seed=51)
    try:
        eta = synth.gaussian_source(dims, L, seed=52)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=oracle_mod.MR_COLUMN)
        out = np.empty_like(eta)
        p = mb.mbicg_default_params(ncycle=ncycle, nmr=nmr, block=block, mr_mode=mb.MBICG_MR_COLUMN,
                                    prec_sap=mb.MBICG_FP16)
        mb.mbicg_sap_precond(ctx, eta, out, L, kappa, p)
        glob, site = errors(out, ref)
        nround = 2 + 4 * ncycle
        assert glob < nround * U_HALF, glob
        assert site < 2e-2, site
        # the FP16 storage changes the result: it is not the FP32 one
        out32 = np.empty_like(eta)
        p.prec_sap = mb.MBICG_FP32
        mb.mbicg_sap_precond(ctx, eta, out32, L, kappa, p)
        assert errors(out32, ref)[0] < 1e-5 < glob
    finally:
        mb.mbicg_destroy(ctx)


def test_fp16_sap_frozen_replay_of_the_oracles_table(oracle_mod):
    """The solver's preconditioner (frozen step lengths) in FP16 storage,
    given the oracle's own table: the same linear operator up to the FP16
    roundings."""
    dims, block, L, ncycle, nmr, kappa = (16, 16, 16, 16), (8, 8, 8, 8), 12, 2, 4, 0.146
    ctx, U = make_ctx(dims, 0.5, seed=53)
    try:
        nd = int(np.prod(dims)) // int(np.prod(block))
        to = np.full((ncycle, 2, nmr, nd), np.nan, dtype=np.complex128)
        eta = synth.gaussian_source(dims, L, seed=54)
        oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=2, omega_table=to)  # records the table
        eta2 = synth.gaussian_source(dims, L, seed=55)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta2, mr_mode=2, omega_table=to)
        p = mb.mbicg_default_params(ncycle=ncycle, nmr=nmr, block=block, mr_mode=mb.MBICG_MR_FROZEN,
                                    prec_sap=mb.MBICG_FP16)
        out = np.empty_like(eta2)
        tx = to.copy()
        assert mb.mbicg_sap_precond_frozen(ctx, eta2, out, L, kappa, p, tx)
        glob, site = errors(out, ref)
        assert glob < (2 + 4 * ncycle) * U_HALF, glob
        assert site < 2e-2, site
    finally:
        mb.mbicg_destroy(ctx)


def test_fp16_sap_refuses_what_it_cannot_run():
    dims = (8, 8, 8, 8)
    ctx, _ = make_ctx(dims, 0.5, seed=56)
    try:
        eta = synth.gaussian_source(dims, 2, seed=57)
        out = np.empty_like(eta)
        for kw in (dict(block=(2, 2, 2, 2)), dict(block=(4, 4, 4, 4), mr_mode=mb.MBICG_MR_BLOCK)):
            p = mb.mbicg_default_params(ncycle=1, nmr=2, prec_sap=mb.MBICG_FP16,
                                        **{"mr_mode": mb.MBICG_MR_COLUMN, **kw})
            with pytest.raises(mb.MbicgError) as e:
                mb.mbicg_sap_precond(ctx, eta, out, 2, 0.12, p)
            assert e.value.status == mb.MBICG_EINVAL
        p = mb.mbicg_default_params(block=(4, 4, 4, 4), prec_sap=mb.MBICG_FP16, prec_D=mb.MBICG_FP64)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_block_solve(ctx, eta, out, 2, 0.12, 1e-10, p)
    finally:
        mb.mbicg_destroy(ctx)
