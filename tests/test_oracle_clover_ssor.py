"""Pins for the oracle's Sec. 2.2 variants: the clover term of the O(a)-improved
Wilson-Dirac matrix, its Jacobi preconditioning A = T^{-1} D_c, and the SSOR
approximation of the domain inverses inside SAP.

The clover term is pinned by the free field (T = 1), constant abelian fields
in every plane and both orientations (closed form 1 -/+ kappa csw sin(B)
sigma_{mu nu}), Hermiticity, chirality, gauge covariance and gamma5-hermiticity
of D_c.  The SSOR domain solve is pinned against a different formulation of
the same operator: Eisenstat's identity turns the printed form into the
Richardson iteration sum_{j=0}^{N} (1 - W A)^j W with
W = (1 - omega U)^{-1} (1 - omega L)^{-1}, built here from dense hopping
matrices that this file assembles itself from the links.
"""
import numpy as np
import pytest

import synth
from lattice_helpers import (CHIRAL_GAMMA, GAMMA5, coords, dense_operator, domain_colour,
                             domain_index, gauge_transform_block, gauge_transform_links,
                             shift_site)

KAPPA, CSW = 0.12, 1.0


def _sigma(mu, nu):
    g = CHIRAL_GAMMA
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _unit_links(dims):
    V = int(np.prod(dims))
    return np.tile(np.eye(3, dtype=np.complex128), (V, 4, 1, 1))


# ---------------------------------------------------------------------------
# clover term
# ---------------------------------------------------------------------------
def test_clover_free_field_is_identity(oracle_mod):
    dims = (4, 2, 4, 6)
    T = oracle_mod.clover(dims, _unit_links(dims), KAPPA, CSW)
    assert np.array_equal(T, np.tile(np.eye(12, dtype=np.complex128), (T.shape[0], 1, 1)))


@pytest.mark.parametrize("mu,nu", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
@pytest.mark.parametrize("orientation", [+1, -1])
def test_clover_constant_abelian_field(oracle_mod, mu, nu, orientation):
    """Colour-diagonal U(1)^3 links with a constant flux B_a through every
    (mu, nu) plaquette: F_{mu nu} = i diag(sin B_a) and
    T = 1 - kappa csw sin(B) sigma_{mu nu} (flux +B), or + for flux -B.
    orientation +1: U_nu(x) = diag(exp(i B_a x_mu)); -1: U_mu(x) = diag(exp(i B_a x_nu))."""
    dims = (4, 6, 4, 8)
    c = coords(dims)
    U = _unit_links(dims)
    along = mu if orientation > 0 else nu      # the coordinate the phase grows with
    link = nu if orientation > 0 else mu       # the link direction that carries it
    n = np.array([1, -2, 3])
    B = 2 * np.pi * n / dims[along]            # periodic in that direction
    ph = np.exp(1j * np.outer(c[:, along], B))  # (V, 3)
    U[:, link] = ph[:, :, None] * np.eye(3)[None]
    T = oracle_mod.clover(dims, U, KAPPA, CSW)
    sign = -1.0 if orientation > 0 else 1.0
    expect = np.eye(12) + sign * KAPPA * CSW * np.kron(_sigma(mu, nu), np.diag(np.sin(B)))
    assert np.max(np.abs(T - expect[None])) < 1e-14


@pytest.fixture(scope="module")
def rough(oracle_mod):
    dims = (4, 4, 2, 4)
    U = synth.su3_links(dims, 0.5, seed=61)
    T = oracle_mod.clover(dims, U, KAPPA, CSW)
    return dims, U, T


def test_clover_hermitian_and_chiral(rough):
    dims, U, T = rough
    assert np.max(np.abs(T - T.conj().transpose(0, 2, 1))) < 1e-15
    g5 = np.kron(GAMMA5, np.eye(3))
    comm = T @ g5 - g5 @ T
    assert np.max(np.abs(comm)) < 1e-15
    assert np.max(np.abs(T - np.eye(12))) > 1e-2  # the field is not trivial


def test_clover_gauge_covariance(oracle_mod, rough):
    """T[U^g]_x = g_x T[U]_x g_x^dagger (colour index) for a random SU(3) g."""
    dims, U, T = rough
    g = synth.gauge_transform(dims, seed=62)
    Tg = oracle_mod.clover(dims, gauge_transform_links(dims, U, g), KAPPA, CSW)
    G = np.einsum("st,vab->vsatb", np.eye(4), g).reshape(-1, 12, 12)
    expect = G @ T @ G.conj().transpose(0, 2, 1)
    assert np.max(np.abs(Tg - expect)) < 1e-14


def test_clover_inverse(oracle_mod, rough):
    dims, U, T = rough
    Ti = oracle_mod.clover_inverse(T)
    assert np.max(np.abs(T @ Ti - np.eye(12))) < 1e-14


def test_clover_D_gamma5_hermitian(oracle_mod, rough):
    """D_c^dagger = gamma5 D_c gamma5 (T is Hermitian and commutes with gamma5),
    and D_c - D = T - 1 site by site."""
    dims, U, T = rough
    D = dense_operator(lambda v: oracle_mod.apply_clover_D(dims, U, KAPPA, T, v), dims)
    V = int(np.prod(dims))
    G5 = np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    assert np.max(np.abs(D.conj().T - G5 @ D @ G5)) < 1e-14
    Dw = dense_operator(lambda v: oracle_mod.apply_D(dims, U, KAPPA, v), dims)
    diff = (D - Dw).reshape(V, 12, V, 12)
    for s in range(V):
        assert np.max(np.abs(diff[s, :, s] - (T[s] - np.eye(12)))) < 1e-15
    off = diff.copy()
    off[np.arange(V), :, np.arange(V)] = 0
    assert np.max(np.abs(off)) < 1e-15


def test_jacobi_preconditioned_operator(oracle_mod, rough):
    """A = T^{-1} D_c; without T it is the Wilson matrix, bit for bit."""
    dims, U, T = rough
    Ti = np.linalg.inv(T)
    psi = synth.gaussian_source(dims, 3, seed=63)
    out = oracle_mod.apply_A(dims, U, KAPPA, Ti, psi)
    Dc = oracle_mod.apply_clover_D(dims, U, KAPPA, T, psi)
    expect = np.einsum("vrc,vci->vri", Ti, Dc.reshape(-1, 12, 3)).reshape(psi.shape)
    assert np.max(np.abs(out - expect)) < 1e-14
    assert np.array_equal(oracle_mod.apply_A(dims, U, KAPPA, None, psi),
                          oracle_mod.apply_D(dims, U, KAPPA, psi))


# ---------------------------------------------------------------------------
# dense hopping matrices assembled here, independently of the oracle
# ---------------------------------------------------------------------------
def _dense_hops(dims, U):
    """Forward and backward hopping matrices (N x N, N = 12 V):
    (Hf psi)_x = sum_mu (1 - gamma_mu) U_mu(x) psi_{x+mu},
    (Hb psi)_x = sum_mu (1 + gamma_mu) U_mu(x-mu)^dagger psi_{x-mu},
    with a factor -1 on hops across the t boundary."""
    V = int(np.prod(dims))
    c = coords(dims)
    Hf = np.zeros((V, 12, V, 12), dtype=np.complex128)
    Hb = np.zeros_like(Hf)
    one = np.eye(4)
    for mu in range(4):
        fwd, bwd = shift_site(dims, mu, +1), shift_site(dims, mu, -1)
        for x in range(V):
            pf = -1.0 if (mu == 3 and c[x, 3] == dims[3] - 1) else 1.0
            pb = -1.0 if (mu == 3 and c[x, 3] == 0) else 1.0
            Hf[x, :, fwd[x]] += pf * np.kron(one - CHIRAL_GAMMA[mu], U[x, mu])
            Hb[x, :, bwd[x]] += pb * np.kron(one + CHIRAL_GAMMA[mu], U[bwd[x], mu].conj().T)
    return Hf.reshape(12 * V, 12 * V), Hb.reshape(12 * V, 12 * V)


def _site_block_diag(Tinv, V):
    if Tinv is None:
        return np.eye(12 * V)
    M = np.zeros((V, 12, V, 12), dtype=np.complex128)
    M[np.arange(V), :, np.arange(V)] = Tinv
    return M.reshape(12 * V, 12 * V)


def _dense_ssor(Lc, Uc, Acc, nssor, omega):
    """sum_{j=0}^{nssor} (1 - W A)^j W, W = (1 - omega U)^{-1} (1 - omega L)^{-1}."""
    n = Acc.shape[0]
    one = np.eye(n)
    W = np.linalg.inv(one - omega * Uc) @ np.linalg.inv(one - omega * Lc)
    R = one - W @ Acc
    S, P = np.zeros_like(W), one.copy()
    for _ in range(nssor + 1):
        S += P
        P = P @ R
    return S @ W


@pytest.fixture(scope="module")
def ssor_problem(oracle_mod, rough):
    dims, U, T = rough
    block = (2, 2, 1, 2)
    V = int(np.prod(dims))
    Hf, Hb = _dense_hops(dims, U)
    Tinv = np.linalg.inv(T)
    return dict(dims=dims, block=block, U=U, T=T, Tinv=Tinv, V=V, Hf=Hf, Hb=Hb,
                dom=domain_index(dims, block), col=domain_colour(dims, block))


def _colour_blocks(p, Tinv, colour):
    V = p["V"]
    same = np.repeat(p["dom"], 12)[:, None] == np.repeat(p["dom"], 12)[None, :]
    Ti = _site_block_diag(Tinv, V)
    Lfull = KAPPA * Ti @ (p["Hf"] * same)
    Ufull = KAPPA * Ti @ (p["Hb"] * same)
    idx = np.nonzero(np.repeat(p["col"], 12) == colour)[0]
    Lc, Uc = Lfull[np.ix_(idx, idx)], Ufull[np.ix_(idx, idx)]
    Acc = np.eye(len(idx)) - Lc - Uc
    return idx, Lc, Uc, Acc


@pytest.mark.parametrize("clover", [False, True])
def test_dense_hops_match_operator(oracle_mod, ssor_problem, clover):
    """The dense construction above is the oracle's A: 1 - kappa T^{-1}(Hf + Hb);
    its forward part is strictly upper triangular in site order inside a
    domain (x + mu has the larger index), the backward part strictly lower, and
    the colour-diagonal block of A has no coupling between domains."""
    p = ssor_problem
    dims, U = p["dims"], p["U"]
    Tinv = p["Tinv"] if clover else None
    A = dense_operator(lambda v: oracle_mod.apply_A(dims, U, KAPPA, Tinv, v), dims)
    Ti = _site_block_diag(Tinv, p["V"])
    assert np.max(np.abs(A - (np.eye(A.shape[0]) - KAPPA * Ti @ (p["Hf"] + p["Hb"])))) < 1e-14
    for colour in (0, 1):
        idx, Lc, Uc, Acc = _colour_blocks(p, Tinv, colour)
        site = np.repeat(np.arange(p["V"]), 12)[idx]
        later = site[:, None] > site[None, :]
        assert np.max(np.abs(Lc[later | (site[:, None] == site[None, :])])) == 0
        assert np.max(np.abs(Uc[~later])) == 0
        assert np.max(np.abs(A[np.ix_(idx, idx)] - Acc)) < 1e-14


@pytest.mark.parametrize("clover", [False, True])
@pytest.mark.parametrize("nssor,omega", [(0, 1.0), (1, 1.26), (3, 0.8)])
def test_ssor_domains_against_richardson_form(oracle_mod, ssor_problem, clover, nssor, omega):
    p = ssor_problem
    Tinv = p["Tinv"] if clover else None
    psi = synth.gaussian_source(p["dims"], 2, seed=64)
    for colour in (0, 1):
        idx, Lc, Uc, Acc = _colour_blocks(p, Tinv, colour)
        B = _dense_ssor(Lc, Uc, Acc, nssor, omega)
        out = oracle_mod.ssor_domains(p["dims"], p["block"], p["U"], KAPPA, nssor, omega, colour,
                                      psi, Tinv=Tinv)
        flat = out.reshape(-1, 2)
        expect = B @ psi.reshape(-1, 2)[idx]
        assert np.max(np.abs(flat[idx] - expect)) < 1e-13 * np.max(np.abs(expect))
        other = np.setdiff1d(np.arange(flat.shape[0]), idx)
        assert np.max(np.abs(flat[other])) == 0


def test_ssor_converges_to_domain_inverse(oracle_mod, ssor_problem):
    """With many terms the SSOR sum is the exact inverse of the domain matrix
    (the spectral radius of 1 - W A is checked below 1 first)."""
    p = ssor_problem
    idx, Lc, Uc, Acc = _colour_blocks(p, p["Tinv"], 1)
    omega = 1.26
    W = np.linalg.inv(np.eye(len(idx)) - omega * Uc) @ np.linalg.inv(np.eye(len(idx)) - omega * Lc)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(len(idx)) - W @ Acc)))
    assert rho < 0.5
    psi = synth.gaussian_source(p["dims"], 1, seed=65)
    out = oracle_mod.ssor_domains(p["dims"], p["block"], p["U"], KAPPA, 60, omega, 1, psi,
                                  Tinv=p["Tinv"])
    expect = np.linalg.solve(Acc, psi.reshape(-1, 1)[idx])
    assert np.max(np.abs(out.reshape(-1, 1)[idx] - expect)) < 1e-12 * np.max(np.abs(expect))


def test_ssor_sap_single_site_domains(oracle_mod):
    """1^4 domains: L = U = 0, so B = 1 for any nssor and omega, and
    K eta = (eta_E, eta_O - A_OE eta_E)."""
    dims, block = (4, 2, 2, 4), (1, 1, 1, 1)
    U = synth.su3_links(dims, 0.5, seed=66)
    eta = synth.gaussian_source(dims, 2, seed=67)
    col = domain_colour(dims, block)
    psi = oracle_mod.sap_ext(dims, block, U, KAPPA, 1, eta, nssor=2, omega=1.26)
    eta_E = eta * (col == 0)[:, None, None, None]
    A_eta_E = oracle_mod.apply_D(dims, U, KAPPA, eta_E)
    expect = np.where((col == 0)[:, None, None, None], eta, eta - A_eta_E)
    assert np.max(np.abs(psi - expect)) < 1e-14


@pytest.mark.parametrize("clover", [False, True])
@pytest.mark.parametrize("ncycle", [1, 2])
def test_ssor_sap_dense_formula(oracle_mod, ssor_problem, clover, ncycle):
    """M_SAP = K sum_{j=0}^{ncycle-1} (1 - A K)^j with B_EE, B_OO the dense SSOR
    matrices (nssor 1, omega 1.26)."""
    p = ssor_problem
    dims, U = p["dims"], p["U"]
    Tinv = p["Tinv"] if clover else None
    A = dense_operator(lambda v: oracle_mod.apply_A(dims, U, KAPPA, Tinv, v), dims)
    N = A.shape[0]
    iE, _, _, _ = _colour_blocks(p, Tinv, 0)
    iO, _, _, _ = _colour_blocks(p, Tinv, 1)
    BEE = _dense_ssor(*_colour_blocks(p, Tinv, 0)[1:], 1, 1.26)
    BOO = _dense_ssor(*_colour_blocks(p, Tinv, 1)[1:], 1, 1.26)
    K = np.zeros((N, N), dtype=np.complex128)
    K[np.ix_(iE, iE)] = BEE
    K[np.ix_(iO, iO)] = BOO
    K[np.ix_(iO, iE)] = -BOO @ A[np.ix_(iO, iE)] @ BEE
    S, P = np.zeros_like(K), np.eye(N, dtype=np.complex128)
    for _ in range(ncycle):
        S += P
        P = P @ (np.eye(N) - A @ K)
    M = K @ S
    eta = synth.gaussian_source(dims, 2, seed=68)
    psi = oracle_mod.sap_ext(dims, p["block"], U, KAPPA, ncycle, eta, Tinv=Tinv, nssor=1,
                             omega=1.26)
    expect = M @ eta.reshape(N, 2)
    assert np.max(np.abs(psi.reshape(N, 2) - expect)) < 1e-13 * np.max(np.abs(expect))


def test_ssor_sap_is_linear_and_column_independent(oracle_mod, ssor_problem):
    """With SSOR domain solves M_SAP is one linear operator (the stationary
    preconditioner Algorithm 1 needs): superposition holds and a column's
    result does not depend on the other columns of the block."""
    p = ssor_problem
    dims, U = p["dims"], p["U"]
    e = synth.gaussian_source(dims, 2, seed=69)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    comb = (a * e[..., 0] + b * e[..., 1])[..., None]
    M = lambda v: oracle_mod.sap_ext(dims, p["block"], U, KAPPA, 2, v, Tinv=p["Tinv"])
    both = M(e)
    assert np.max(np.abs(M(comb)[..., 0] - (a * both[..., 0] + b * both[..., 1]))) < 1e-13
    assert np.max(np.abs(M(e[..., :1])[..., 0] - both[..., 0])) < 1e-15


def test_ssor_sap_gauge_covariance(oracle_mod, ssor_problem):
    p = ssor_problem
    dims, U = p["dims"], p["U"]
    g = synth.gauge_transform(dims, seed=70)
    Ug = gauge_transform_links(dims, U, g)
    Tg = oracle_mod.clover(dims, Ug, KAPPA, CSW)
    eta = synth.gaussian_source(dims, 2, seed=71)
    psi = oracle_mod.sap_ext(dims, p["block"], U, KAPPA, 2, eta, Tinv=p["Tinv"])
    psig = oracle_mod.sap_ext(dims, p["block"], Ug, KAPPA, 2, gauge_transform_block(g, eta),
                              Tinv=np.linalg.inv(Tg))
    assert np.max(np.abs(psig - gauge_transform_block(g, psi))) < 1e-13


def test_ssor_argument_errors(oracle_mod, ssor_problem):
    p = ssor_problem
    psi = synth.gaussian_source(p["dims"], 1, seed=72)
    for nssor, omega, colour in [(-1, 1.0, 0), (1, 0.0, 0), (1, 2.0, 0), (1, 1.0, 2)]:
        with pytest.raises(ValueError):
            oracle_mod.ssor_domains(p["dims"], p["block"], p["U"], KAPPA, nssor, omega, colour, psi)
    with pytest.raises(ValueError):
        oracle_mod.sap_ext(p["dims"], (4, 4, 2, 4), p["U"], KAPPA, 1, psi)  # one domain per direction


# ---------------------------------------------------------------------------
# the block solve with the Sec. 2.2 variants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("clover,solver", [(False, 1), (True, 1), (True, 0)])
def test_block_solve_variants_match_dense(oracle_mod, ssor_problem, clover, solver):
    """Algorithm 1 with SAP (SSOR or frozen-MR domain solves) on the Wilson or
    the Jacobi-preconditioned clover matrix: D X = B solved through A X = T^{-1} B
    agrees with a dense LAPACK solve of D X = B."""
    p = ssor_problem
    dims, U, T = p["dims"], p["U"], p["T"]
    V = p["V"]
    B = synth.gaussian_source(dims, 3, seed=73)
    if clover:
        Tinv = p["Tinv"]
        D = dense_operator(lambda v: oracle_mod.apply_clover_D(dims, U, KAPPA, T, v), dims)
        Bp = np.einsum("vrc,vci->vri", Tinv, B.reshape(V, 12, 3)).reshape(B.shape)
    else:
        Tinv = None
        D = dense_operator(lambda v: oracle_mod.apply_D(dims, U, KAPPA, v), dims)
        Bp = B
    res = oracle_mod.block_bicgstab(dims, U, KAPPA, Bp, 1e-12, max_iter=200, ncycle=2,
                                    nmr=4, block=p["block"], mr_mode=oracle_mod.MR_FROZEN,
                                    Tinv=Tinv, solver=solver, nssor=1, omega=1.26)
    assert res["status"] == 0 and np.max(res["true_res"]) <= 1e-11
    X = np.linalg.solve(D, B.reshape(-1, 3))
    err = np.linalg.norm(res["X"].reshape(-1, 3) - X, axis=0) / np.linalg.norm(X, axis=0)
    assert np.max(err) < 1e-9
