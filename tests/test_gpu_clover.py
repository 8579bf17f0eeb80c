"""Parity of the clover term and its Jacobi preconditioning (Sec. 2.2) on the
GPU with the FP64 oracle, through the C ABI: the clover matrix D_c and the
Jacobi-preconditioned A = T^{-1} D_c (1e-13 per-site in FP64, 1e-6 in FP32),
SAP on A (FP64 and FP32), and the block solve of D_c X = B against a dense
solve and the oracle's operator."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx, rel_col_norm, rel_site_norm
from lattice_helpers import dense_operator

pytestmark = pytest.mark.gpu

CSW = 1.3


@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 4), ((6, 2, 4, 10), 12), ((8, 4, 2, 2), 16)])
def test_clover_operators_match_oracle(oracle_mod, dims, L):
    ctx, U = make_ctx(dims, 0.5, seed=41)
    try:
        kappa = 0.125
        mb.mbicg_load_clover(ctx, CSW)
        T = oracle_mod.clover(dims, U, kappa, CSW)
        Ti = oracle_mod.clover_inverse(T)
        psi = synth.gaussian_source(dims, L, seed=42)
        out = np.empty_like(psi)
        ref_c = oracle_mod.apply_clover_D(dims, U, kappa, T, psi)
        ref_a = oracle_mod.apply_A(dims, U, kappa, Ti, psi)
        for prec, tol in ((mb.MBICG_FP64, 1e-13), (mb.MBICG_FP32, 1e-6)):
            mb.mbicg_apply_clover(ctx, psi, out, L, kappa, prec, 0)
            assert rel_site_norm(out, ref_c) < tol
            mb.mbicg_apply_clover(ctx, psi, out, L, kappa, prec, 1)
            assert rel_site_norm(out, ref_a) < tol
        # a new kappa forms a new T^{-1}
        k2 = 0.131
        mb.mbicg_apply_clover(ctx, psi, out, L, k2, mb.MBICG_FP64, 1)
        Ti2 = oracle_mod.clover_inverse(oracle_mod.clover(dims, U, k2, CSW))
        assert rel_site_norm(out, oracle_mod.apply_A(dims, U, k2, Ti2, psi)) < 1e-13
        # csw = 0: the clover matrix is the Wilson matrix
        mb.mbicg_load_clover(ctx, 0.0)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_apply_clover(ctx, psi, out, L, kappa, mb.MBICG_FP64, 0)
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.parametrize("prec,tol,mode", [(mb.MBICG_FP64, 1e-12, 0), (mb.MBICG_FP64, 1e-12, 1),
                                           (mb.MBICG_FP32, 1e-5, 0)])
def test_clover_sap_matches_oracle(oracle_mod, prec, tol, mode):
    dims, block, L = (8, 4, 4, 8), (4, 2, 2, 4), 3
    ctx, U = make_ctx(dims, 0.5, seed=43)
    try:
        kappa = 0.125
        mb.mbicg_load_clover(ctx, CSW)
        Ti = oracle_mod.clover_inverse(oracle_mod.clover(dims, U, kappa, CSW))
        eta = synth.gaussian_source(dims, L, seed=44)
        p = mb.mbicg_default_params(ncycle=2, nmr=3, block=block, mr_mode=mode, prec_sap=prec, clover=1)
        out = np.empty_like(eta)
        mb.mbicg_sap_precond(ctx, eta, out, L, kappa, p)
        ref = oracle_mod.sap_ext(dims, block, U, kappa, 2, eta, Tinv=Ti, solver=oracle_mod.DOMAIN_MR, nmr=3,
                                 mr_mode=mode)
        assert rel_site_norm(out, ref) < tol
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.parametrize("prec_D", [mb.MBICG_FP64, mb.MBICG_FP32])
def test_clover_block_solve(oracle_mod, prec_D):
    """D_c X = B through A X = T^{-1} B with SAP on A: X against a dense LAPACK
    solve of D_c X = B, and the residual of D_c with the oracle's operator."""
    dims, block, L = (4, 4, 2, 4), (2, 2, 1, 2), 3
    ctx, U = make_ctx(dims, 0.5, seed=45)
    try:
        kappa = 0.12
        mb.mbicg_load_clover(ctx, CSW)
        T = oracle_mod.clover(dims, U, kappa, CSW)
        B = synth.gaussian_source(dims, L, seed=46)
        p = mb.mbicg_default_params(ncycle=2, nmr=4, block=block, prec_D=prec_D, clover=1)
        X = np.empty_like(B)
        st, iters, tres = mb.mbicg_block_solve(ctx, B, X, L, kappa, 1e-11, p)
        assert st == mb.MBICG_OK and max(tres) <= 1e-11
        D = dense_operator(lambda v: oracle_mod.apply_clover_D(dims, U, kappa, T, v), dims)
        Xd = np.linalg.solve(D, B.reshape(-1, L)).reshape(B.shape)
        assert rel_col_norm(X, Xd) < 1e-8
        R = B - oracle_mod.apply_clover_D(dims, U, kappa, T, X)
        rel = np.linalg.norm(R.reshape(-1, L), axis=0) / np.linalg.norm(B.reshape(-1, L), axis=0)
        assert rel.max() < 1e-9
    finally:
        mb.mbicg_destroy(ctx)


def test_clover_errors():
    dims = (4, 4, 4, 4)
    ctx = mb.mbicg_create(dims)
    try:
        psi = synth.gaussian_source(dims, 1, seed=47)
        out = np.empty_like(psi)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_load_clover(ctx, CSW)            # no gauge field
        mb.mbicg_load_gauge(ctx, synth.su3_links(dims, 0.5, seed=48))
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(mb.MbicgError):
                mb.mbicg_load_clover(ctx, bad)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_apply_clover(ctx, psi, out, 1, 0.12, mb.MBICG_FP64, 0)  # no clover term
        mb.mbicg_load_clover(ctx, CSW)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_apply_clover(ctx, psi, out, 1, 0.12, mb.MBICG_FP16, 0)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_apply_clover(ctx, psi, out, 1, 0.12, mb.MBICG_FP64, 2)
        # a new gauge field switches the clover term off
        mb.mbicg_load_gauge(ctx, synth.su3_links(dims, 0.5, seed=49))
        with pytest.raises(mb.MbicgError):
            mb.mbicg_apply_clover(ctx, psi, out, 1, 0.12, mb.MBICG_FP64, 1)
        p = mb.mbicg_default_params(ncycle=1, nmr=2, block=(2, 2, 2, 2), clover=1)
        X = np.empty_like(psi)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_block_solve(ctx, psi, X, 1, 0.12, 1e-8, p)
    finally:
        mb.mbicg_destroy(ctx)
