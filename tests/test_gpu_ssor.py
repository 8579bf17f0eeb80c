"""Parity of the SSOR domain solves of Sec. 2.2 on the GPU with the FP64
oracle, through the C ABI: SAP with SSOR domain solves for the Wilson and the
Jacobi-preconditioned clover matrix (FP64 1e-12, FP32 1e-5), its linearity,
and the block solve with it against a dense solve."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx, rel_col_norm, rel_site_norm
from lattice_helpers import dense_operator

pytestmark = pytest.mark.gpu

CSW = 1.3


@pytest.mark.parametrize("dims,block,clover", [((8, 4, 4, 8), (4, 2, 2, 4), False),
                                               ((8, 4, 4, 8), (4, 2, 2, 4), True),
                                               ((16, 8, 8, 8), (8, 4, 4, 4), False)])
@pytest.mark.parametrize("prec,tol", [(mb.MBICG_FP64, 1e-12), (mb.MBICG_FP32, 1e-5)])
def test_ssor_sap_matches_oracle(oracle_mod, dims, block, clover, prec, tol):
    L, kappa = 3, 0.125
    ctx, U = make_ctx(dims, 0.5, seed=51)
    try:
        Ti = None
        if clover:
            mb.mbicg_load_clover(ctx, CSW)
            Ti = oracle_mod.clover_inverse(oracle_mod.clover(dims, U, kappa, CSW))
        eta = synth.gaussian_source(dims, L, seed=52)
        p = mb.mbicg_default_params(ncycle=2, block=block, prec_sap=prec, clover=int(clover),
                                    domain_solver=mb.MBICG_DOMAIN_SSOR, nssor=1, ssor_omega=1.26)
        out = np.empty_like(eta)
        mb.mbicg_sap_precond(ctx, eta, out, L, kappa, p)
        ref = oracle_mod.sap_ext(dims, block, U, kappa, 2, eta, Tinv=Ti, solver=oracle_mod.DOMAIN_SSOR,
                                 nssor=1, omega=1.26)
        assert rel_site_norm(out, ref) < tol
    finally:
        mb.mbicg_destroy(ctx)


def test_ssor_sap_is_linear():
    """SSOR domain solves make M_SAP one linear operator: superposition holds
    and a column's result does not depend on the other columns."""
    dims, block = (8, 4, 4, 8), (4, 2, 2, 4)
    ctx, U = make_ctx(dims, 0.5, seed=53)
    try:
        e = synth.gaussian_source(dims, 2, seed=54)
        p = mb.mbicg_default_params(ncycle=2, block=block, prec_sap=mb.MBICG_FP64,
                                    domain_solver=mb.MBICG_DOMAIN_SSOR)
        both = np.empty_like(e)
        mb.mbicg_sap_precond(ctx, e, both, 2, 0.125, p)
        a, b = 0.7 - 0.2j, -1.3 + 0.5j
        comb = np.ascontiguousarray((a * e[..., 0] + b * e[..., 1])[..., None])
        out = np.empty_like(comb)
        mb.mbicg_sap_precond(ctx, comb, out, 1, 0.125, p)
        assert rel_site_norm(out[..., 0:1], (a * both[..., 0] + b * both[..., 1])[..., None]) < 1e-12
        one = np.empty_like(comb)
        mb.mbicg_sap_precond(ctx, np.ascontiguousarray(e[..., :1]), one, 1, 0.125, p)
        assert rel_site_norm(one, np.ascontiguousarray(both[..., :1])) < 1e-14
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.parametrize("clover,prec_D", [(False, mb.MBICG_FP64), (False, mb.MBICG_FP32), (True, mb.MBICG_FP32)])
def test_ssor_block_solve(oracle_mod, clover, prec_D):
    dims, block, L, kappa = (4, 4, 2, 4), (2, 2, 1, 2), 3, 0.12
    ctx, U = make_ctx(dims, 0.5, seed=55)
    try:
        if clover:
            mb.mbicg_load_clover(ctx, CSW)
            T = oracle_mod.clover(dims, U, kappa, CSW)
            op = lambda v: oracle_mod.apply_clover_D(dims, U, kappa, T, v)
        else:
            op = lambda v: oracle_mod.apply_D(dims, U, kappa, v)
        B = synth.gaussian_source(dims, L, seed=56)
        p = mb.mbicg_default_params(ncycle=2, block=block, prec_D=prec_D, clover=int(clover),
                                    domain_solver=mb.MBICG_DOMAIN_SSOR)
        X = np.empty_like(B)
        st, iters, tres = mb.mbicg_block_solve(ctx, B, X, L, kappa, 1e-11, p)
        assert st == mb.MBICG_OK and max(tres) <= 1e-11
        # SSOR makes M one linear operator: the iteration graph is used from the start
        assert mb.mbicg_get_stats(ctx)["graph_iterations"] >= 1
        Xd = np.linalg.solve(dense_operator(op, dims), B.reshape(-1, L)).reshape(B.shape)
        assert rel_col_norm(X, Xd) < 1e-8
    finally:
        mb.mbicg_destroy(ctx)


def test_ssor_params_errors():
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(dims, 0.5, seed=57)
    try:
        e = synth.gaussian_source(dims, 1, seed=58)
        out = np.empty_like(e)
        for kw in (dict(nssor=-1), dict(nssor=17), dict(ssor_omega=0.0), dict(ssor_omega=2.0),
                   dict(domain_solver=2)):
            args = dict(ncycle=1, block=(2, 2, 2, 2), domain_solver=mb.MBICG_DOMAIN_SSOR)
            args.update(kw)
            with pytest.raises(mb.MbicgError):
                mb.mbicg_sap_precond(ctx, e, out, 1, 0.12, mb.mbicg_default_params(**args))
    finally:
        mb.mbicg_destroy(ctx)
