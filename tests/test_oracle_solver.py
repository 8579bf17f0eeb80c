"""Pins for the oracle's QR, L x L solves and modified block BiCGSTAB
(Algorithm 1, Sec. 2.1).

Checks from outside the oracle: Q^H Q = 1 and P = Q gamma with the unique
positive-diagonal gamma (compared with LAPACK's QR after fixing phases), LU
against numpy.linalg.solve, the solution against a dense LAPACK solve on 2^4
and 4^4 lattices, L = 1 against textbook right-preconditioned BiCGSTAB
(van der Vorst 1992), and Algorithm 2 (the memory-saving form) written
independently with dense matrices.
"""
import numpy as np
import pytest

import synth
from lattice_helpers import dense_operator


def test_qr_mgs_properties(oracle_mod):
    rng = np.random.default_rng(3)
    P = rng.standard_normal((500, 7)) + 1j * rng.standard_normal((500, 7))
    Q, g = oracle_mod.qr_mgs(P)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(7))) < 1e-14
    assert np.max(np.abs(Q @ g - P)) < 1e-14 * np.max(np.abs(P))
    assert np.all(np.tril(g, -1) == 0)
    assert np.all(np.abs(np.diag(g).imag) == 0) and np.all(np.diag(g).real > 0)
    # uniqueness: LAPACK's QR with its diagonal phases removed gives the same Q
    Ql, Rl = np.linalg.qr(P)
    ph = np.diag(Rl) / np.abs(np.diag(Rl))
    assert np.max(np.abs(Ql * ph[None, :] - Q)) < 1e-13
    assert np.max(np.abs(Rl / ph[:, None] - g)) < 1e-12


def test_qr_mgs_rank_deficient(oracle_mod):
    rng = np.random.default_rng(4)
    P = rng.standard_normal((50, 3)) + 0j
    P[:, 2] = 2 * P[:, 0] - P[:, 1]
    P[:, 2] += 0  # exactly dependent only up to rounding; make it exact below
    P2 = np.zeros((50, 3), dtype=np.complex128)
    P2[:, 0] = P[:, 0]
    P2[:, 1] = P[:, 0]  # identical column: MGS leaves an exact zero
    with pytest.raises(np.linalg.LinAlgError):
        oracle_mod.qr_mgs(P2)


def test_lu_solve(oracle_mod):
    rng = np.random.default_rng(5)
    for L in (1, 4, 12):
        G = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
        C = rng.standard_normal((L, 3)) + 1j * rng.standard_normal((L, 3))
        X = oracle_mod.lu_solve(G, C)
        assert np.max(np.abs(X - np.linalg.solve(G, C))) < 1e-12
    # a matrix that needs pivoting (zero leading entry)
    G = np.array([[0, 1, 0], [1, 0, 0], [0, 0, 2]], dtype=np.complex128)
    C = np.eye(3, dtype=np.complex128)
    assert np.allclose(oracle_mod.lu_solve(G, C), np.linalg.inv(G), atol=1e-15)
    with pytest.raises(np.linalg.LinAlgError):
        oracle_mod.lu_solve(np.zeros((2, 2)), np.eye(2))


@pytest.mark.parametrize("dims,block,L,ncycle", [
    ((2, 2, 2, 2), (1, 1, 1, 1), 3, 2),
    ((4, 4, 4, 4), (2, 2, 2, 2), 4, 4),
    ((4, 4, 4, 4), None, 4, 0),
])
def test_block_solve_matches_dense_lu(oracle_mod, dims, block, L, ncycle):
    """The converged X equals the dense LAPACK solution of A X = B."""
    U = synth.su3_links(dims, 0.4, seed=1000)
    kappa = 0.12
    B = synth.gaussian_source(dims, L, seed=2000)
    res = oracle_mod.block_bicgstab(dims, U, kappa, B, tol=1e-12, max_iter=500,
                                    ncycle=ncycle, nmr=4, block=block)
    assert res["status"] == 0
    assert res["true_res"].max() < 1e-11
    A = dense_operator(lambda v: oracle_mod.apply_D(dims, U, kappa, v), dims)
    N = A.shape[0]
    Xd = np.linalg.solve(A, B.reshape(N, L))
    cond = np.linalg.cond(A)
    err = np.linalg.norm(res["X"].reshape(N, L) - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
    assert err.max() < 10 * cond * 1e-12
    # recursive and true residuals agree at convergence
    assert res["history"][-1] <= 1e-12
    assert res["true_res"].max() < 10 * 1e-12


def _textbook_bicgstab(Aop, Mop, b, iters):
    """Right-preconditioned BiCGSTAB (van der Vorst 1992) for one vector."""
    x = np.zeros_like(b)
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = []
    for _ in range(iters):
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        y = Mop(p)
        v = Aop(y)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        z = Mop(s)
        t = Aop(z)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * y + omega * z
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / np.linalg.norm(b))
    return x, np.array(hist)


@pytest.mark.parametrize("ncycle", [0, 2])
def test_L1_reduces_to_textbook_bicgstab(oracle_mod, ncycle):
    dims, block = (4, 4, 2, 4), (2, 2, 1, 2)
    U = synth.su3_links(dims, 0.5, seed=101)
    kappa = 0.125
    b = synth.gaussian_source(dims, 1, seed=102)
    Aop = lambda v: oracle_mod.apply_D(dims, U, kappa, v)
    Mop = (lambda v: v) if ncycle == 0 else (
        lambda v: oracle_mod.sap(dims, block, U, kappa, ncycle, 3, v))
    n = 15
    x_tb, h_tb = _textbook_bicgstab(Aop, Mop, b, n)
    res = oracle_mod.block_bicgstab(dims, U, kappa, b, tol=1e-300, max_iter=n,
                                    ncycle=ncycle, nmr=3, block=block)
    assert res["iters"] == n and res["status"] == 1
    # the two recursions agree to rounding, relative to the residual level reached
    assert np.max(np.abs(res["history"] - h_tb) / h_tb) < 1e-8
    assert np.max(np.abs(res["X"] - x_tb)) < 1e-8 * np.max(np.abs(x_tb))


def test_algorithm2_equals_algorithm1(oracle_mod):
    """Algorithm 2 (memory saving) written with dense matrices gives the same
    iterates as the oracle's Algorithm 1 with M = 1."""
    dims = (2, 2, 2, 4)
    U = synth.su3_links(dims, 0.5, seed=111)
    kappa = 0.125
    L = 3
    B = synth.gaussian_source(dims, L, seed=112)
    A = dense_operator(lambda v: oracle_mod.apply_D(dims, U, kappa, v), dims)
    N = A.shape[0]
    Bm = B.reshape(N, L)
    X = np.zeros_like(Bm)
    R = Bm - A @ X
    P = R.copy()
    Rt = R.copy()
    hist = []
    for _ in range(8):
        P, _ = np.linalg.qr(P)  # any orthonormal basis of span(P) gives the same X, R
        Ub = P
        Vb = A @ Ub
        G = Rt.conj().T @ Vb
        alpha = np.linalg.solve(G, Rt.conj().T @ R)
        R = R - Vb @ alpha
        X = X + Ub @ alpha
        S = R
        Z = A @ S
        zeta = np.trace(Z.conj().T @ R) / np.trace(Z.conj().T @ Z)
        X = X + zeta * S
        R = R - zeta * Z
        beta = np.linalg.solve(G, -(Rt.conj().T @ Z))
        P = R + (P - zeta * Vb) @ beta
        hist.append(np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(Bm, axis=0)))
    res = oracle_mod.block_bicgstab(dims, U, kappa, B, tol=1e-300, max_iter=8)
    assert np.max(np.abs(res["history"] - np.array(hist)) / np.array(hist)) < 1e-9
    assert np.max(np.abs(res["X"].reshape(N, L) - X)) < 1e-9 * np.max(np.abs(X))


@pytest.mark.parametrize("ncycle", [0, 2])
@pytest.mark.parametrize("delta", [1e-6, 1e-10])
def test_qr_keeps_true_residual_with_nearly_dependent_columns(oracle_mod, ncycle, delta):
    """Sec. 2.1: the QR of P is there for numerical accuracy (in exact
    arithmetic P -> P gamma^{-1} only rescales alpha and beta, and the
    residuals are unchanged).  With right-hand sides that differ by delta the
    unorthogonalised block becomes nearly rank deficient and the recursive
    residual drifts away from the true one (true residual 1e-9 .. 1e-6 at a
    recursive 1e-12 when the QR is left out); with the QR both stay together."""
    dims = (4, 4, 4, 4)
    U = synth.su3_links(dims, 0.4, seed=1000)
    B = synth.gaussian_source(dims, 4, seed=5)
    rng = np.random.default_rng(3)
    for i in range(1, 4):
        B[..., i] = B[..., 0] + delta * (rng.standard_normal(B.shape[:3])
                                         + 1j * rng.standard_normal(B.shape[:3]))
    rt = synth.gaussian_source(dims, 4, seed=9)
    res = oracle_mod.block_bicgstab(dims, U, 0.12, B, 1e-12, max_iter=300, ncycle=ncycle, nmr=4,
                                    block=(2, 2, 2, 2), mr_mode=oracle_mod.MR_FROZEN, rtilde=rt)
    assert res["status"] == 0
    assert np.max(res["true_res"]) < 1e-11


def test_block_solve_statuses(oracle_mod):
    dims = (2, 2, 2, 2)
    U = synth.su3_links(dims, 0.4, seed=1)
    B = synth.gaussian_source(dims, 2, seed=2)
    # not converged within max_iter
    res = oracle_mod.block_bicgstab(dims, U, 0.12, B, tol=1e-14, max_iter=2)
    assert res["status"] == 1 and res["iters"] == 2
    # a zero shadow block makes R~^H V singular: breakdown
    res = oracle_mod.block_bicgstab(dims, U, 0.12, B, tol=1e-14, max_iter=5,
                                    rtilde=np.zeros_like(B))
    assert res["status"] == 2
    # a zero right-hand side column is rejected
    B0 = B.copy()
    B0[..., 1] = 0
    with pytest.raises(ValueError):
        oracle_mod.block_bicgstab(dims, U, 0.12, B0, tol=1e-10)


def test_iterations_fall_with_block_size(oracle_mod):
    """Sec. 3.3 and Table 1: larger L needs fewer iterations.  Qualitative only
    (the paper's gauge fields are not available).  With the stationary (frozen
    step length) SAP the block method keeps the trend of the paper; with
    per-column MR step lengths M is not a fixed linear operator and the gain
    is lost, which is why Sec. 2.1 asks for a stationary M."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synth.su3_links(dims, 0.5, seed=1001)
    kappa = 0.16
    B = synth.gaussian_source(dims, 8, seed=2001)
    it = {}
    for L in (1, 8):
        worst = 0
        for j in range(0, 8, L):
            r = oracle_mod.block_bicgstab(dims, U, kappa, B[..., j:j + L], tol=1e-10,
                                          max_iter=1000, ncycle=1, nmr=4, block=block,
                                          mr_mode=2)
            assert r["status"] == 0 and r["true_res"].max() < 1e-9
            worst = max(worst, r["iters"])
        it[L] = worst
    assert it[8] < 0.75 * it[1]
