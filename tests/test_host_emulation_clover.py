"""The clover term, its Jacobi preconditioning and the SSOR domain solves of
Sec. 2.2 through the C ABI on the CPU: the emulated library (built by
tests/emulated_library.py from the CUDA sources; host code and kernels the
library's own) against the FP64 oracle.  Covers mbicg_load_clover,
mbicg_apply_clover (D_c and A = T^{-1} D_c, FP64 and FP32, a change of
kappa), mbicg_sap_precond with MR and SSOR domain solves on the Wilson and
the clover matrix, mbicg_block_solve of D_c X = B, and the argument errors."""
import ctypes

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb  # the ctypes structures only; no library is loaded
import synth

DIMS, L, KAPPA, CSW = (4, 4, 4, 4), 2, 0.125, 1.3


def _v(a):
    return ctypes.c_void_p(a.ctypes.data)


def _rel_site(a, b):
    """Largest per-site spinor-norm difference over the largest site norm."""
    d = np.linalg.norm((a - b).reshape(a.shape[0], -1, a.shape[3]), axis=1)
    return float(d.max() / np.linalg.norm(b.reshape(b.shape[0], -1, b.shape[3]), axis=1).max())


@pytest.fixture(scope="module")
def lib(emulated_library):
    lb = emulated_library
    lb.mbicg_load_clover.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lb.mbicg_apply_clover.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int]
    return lb


@pytest.fixture(scope="module")
def ctx(lib):
    c = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(c), (ctypes.c_int * 4)(*DIMS), 0, None) == mb.MBICG_OK
    U = synth.su3_links(DIMS, 0.5, seed=1100)
    assert lib.mbicg_load_gauge(c, _v(U)) == mb.MBICG_OK
    assert lib.mbicg_load_clover(c, CSW) == mb.MBICG_OK
    yield c, U
    lib.mbicg_destroy(c)


@pytest.fixture(scope="module")
def terms(oracle_mod, ctx):
    T = oracle_mod.clover(DIMS, ctx[1], KAPPA, CSW)
    return T, oracle_mod.clover_inverse(T)


def _params(lib, **kw):
    p = mb.mbicg_params()
    lib.mbicg_default_params(ctypes.byref(p))
    p.block = (ctypes.c_int * 4)(2, 2, 2, 2)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("prec,tol", [(mb.MBICG_FP64, 1e-13), (mb.MBICG_FP32, 1e-6)])
def test_clover_operators(lib, ctx, terms, oracle_mod, prec, tol):
    c, U = ctx
    T, Ti = terms
    psi = synth.gaussian_source(DIMS, L, seed=1101)
    out = np.empty_like(psi)
    assert lib.mbicg_apply_clover(c, _v(psi), _v(out), L, KAPPA, prec, 0) == mb.MBICG_OK
    assert _rel_site(out, oracle_mod.apply_clover_D(DIMS, U, KAPPA, T, psi)) < tol
    assert lib.mbicg_apply_clover(c, _v(psi), _v(out), L, KAPPA, prec, 1) == mb.MBICG_OK
    assert _rel_site(out, oracle_mod.apply_A(DIMS, U, KAPPA, Ti, psi)) < tol
    # another kappa forms another T^{-1}; then back
    k2 = 0.131
    assert lib.mbicg_apply_clover(c, _v(psi), _v(out), L, k2, prec, 1) == mb.MBICG_OK
    Ti2 = oracle_mod.clover_inverse(oracle_mod.clover(DIMS, U, k2, CSW))
    assert _rel_site(out, oracle_mod.apply_A(DIMS, U, k2, Ti2, psi)) < tol
    assert lib.mbicg_apply_clover(c, _v(psi), _v(out), L, KAPPA, prec, 1) == mb.MBICG_OK
    assert _rel_site(out, oracle_mod.apply_A(DIMS, U, KAPPA, Ti, psi)) < tol


@pytest.mark.parametrize("clover,solver,prec,tol", [
    (1, 0, mb.MBICG_FP64, 1e-12), (1, 0, mb.MBICG_FP32, 1e-5),
    (0, 1, mb.MBICG_FP64, 1e-12), (0, 1, mb.MBICG_FP32, 1e-5),
    (1, 1, mb.MBICG_FP64, 1e-12), (1, 1, mb.MBICG_FP32, 1e-5)])
def test_sap_domain_solvers(lib, ctx, terms, oracle_mod, clover, solver, prec, tol):
    c, U = ctx
    Ti = terms[1] if clover else None
    eta = synth.gaussian_source(DIMS, L, seed=1102)
    out = np.empty_like(eta)
    p = _params(lib, ncycle=2, nmr=3, mr_mode=mb.MBICG_MR_COLUMN, prec_sap=prec, clover=clover,
                domain_solver=solver, nssor=2, ssor_omega=1.2)
    assert lib.mbicg_sap_precond(c, _v(eta), _v(out), L, KAPPA, ctypes.byref(p)) == mb.MBICG_OK, \
        lib.mbicg_last_error(c)
    ref = oracle_mod.sap_ext(DIMS, (2, 2, 2, 2), U, KAPPA, 2, eta, Tinv=Ti, solver=solver, nmr=3,
                             mr_mode=oracle_mod.MR_COLUMN, nssor=2, omega=1.2)
    assert _rel_site(out, ref) < tol


@pytest.mark.parametrize("solver", [0, 1])
def test_clover_block_solve(lib, ctx, terms, oracle_mod, solver):
    """D_c X = B, solved as A X = T^{-1} B, with MR or SSOR domain solves: the
    residual of D_c with the oracle's operator."""
    c, U = ctx
    T = terms[0]
    B = synth.gaussian_source(DIMS, L, seed=1103)
    X = np.empty_like(B)
    p = _params(lib, ncycle=2, nmr=4, clover=1, domain_solver=solver)
    it = ctypes.c_int(0)
    tres = np.zeros(L)
    rc = lib.mbicg_block_solve(c, _v(B), _v(X), L, KAPPA, 1e-10, ctypes.byref(p), ctypes.byref(it),
                               tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == mb.MBICG_OK and it.value > 0, lib.mbicg_last_error(c)
    assert tres.max() <= 1e-10
    R = B - oracle_mod.apply_clover_D(DIMS, U, KAPPA, T, X)
    rel = np.linalg.norm(R.reshape(-1, L), axis=0) / np.linalg.norm(B.reshape(-1, L), axis=0)
    # true_res refers to A X = T^{-1} B; D_c = T A, with T close to 1
    assert rel.max() < 1e-9


def test_clover_argument_errors(lib, oracle_mod):
    c = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(c), (ctypes.c_int * 4)(*DIMS), 0, None) == mb.MBICG_OK
    try:
        psi = synth.gaussian_source(DIMS, 1, seed=1104)
        out = np.empty_like(psi)
        assert lib.mbicg_load_clover(c, CSW) == mb.MBICG_ENOGAUGE
        assert lib.mbicg_load_gauge(c, _v(synth.su3_links(DIMS, 0.5, seed=1105))) == mb.MBICG_OK
        for bad in (-1.0, float("nan"), float("inf")):
            assert lib.mbicg_load_clover(c, bad) == mb.MBICG_EINVAL
        assert lib.mbicg_apply_clover(c, _v(psi), _v(out), 1, KAPPA, mb.MBICG_FP64, 0) == mb.MBICG_EINVAL
        assert lib.mbicg_load_clover(c, CSW) == mb.MBICG_OK
        assert lib.mbicg_apply_clover(c, _v(psi), _v(out), 1, KAPPA, mb.MBICG_FP16, 0) == mb.MBICG_EINVAL
        assert lib.mbicg_apply_clover(c, _v(psi), _v(out), 1, KAPPA, mb.MBICG_FP64, 2) == mb.MBICG_EINVAL
        for kw in (dict(nssor=-1), dict(nssor=17), dict(ssor_omega=0.0), dict(ssor_omega=2.0),
                   dict(domain_solver=2)):
            p = _params(lib, ncycle=1, domain_solver=1, **{k: v for k, v in kw.items() if k != "domain_solver"})
            if "domain_solver" in kw:
                p.domain_solver = kw["domain_solver"]
            assert lib.mbicg_sap_precond(c, _v(psi), _v(out), 1, KAPPA, ctypes.byref(p)) == mb.MBICG_EINVAL
        # a new gauge field switches the clover term off
        assert lib.mbicg_load_gauge(c, _v(synth.su3_links(DIMS, 0.5, seed=1106))) == mb.MBICG_OK
        assert lib.mbicg_apply_clover(c, _v(psi), _v(out), 1, KAPPA, mb.MBICG_FP64, 1) == mb.MBICG_EINVAL
        p = _params(lib, ncycle=1, nmr=2, clover=1)
        it = ctypes.c_int(0)
        tres = np.zeros(1)
        assert lib.mbicg_block_solve(c, _v(psi), _v(out), 1, KAPPA, 1e-8, ctypes.byref(p), ctypes.byref(it),
                                     tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == mb.MBICG_EINVAL
    finally:
        lib.mbicg_destroy(c)
