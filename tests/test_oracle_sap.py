"""Pins for the oracle's SAP preconditioner (Sec. 2.2).

M_SAP = K sum_{j=0}^{ncycle-1} (1 - A K)^j with
K = [[B_EE, 0], [-B_OO A_OE B_EE, B_OO]] over checkerboard-coloured domains.
The checks: single-site domains (B = 1 exactly), MR iterated to convergence
against the dense formula with exact block inverses, one MR step against its
closed form on dense domain matrices, and gauge covariance.
"""
import numpy as np
import pytest

import synth
from lattice_helpers import (dense_operator, domain_colour, domain_index,
                             gauge_transform_block, gauge_transform_links)


@pytest.fixture(scope="module")
def small_problem(oracle_mod):
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synth.su3_links(dims, 0.4, seed=1000)
    kappa = 0.12
    A = dense_operator(lambda v: oracle_mod.apply_D(dims, U, kappa, v), dims)
    return dims, block, U, kappa, A


def _dense_sap(A, colour_rows, ncycle):
    """K sum_j (1 - A K)^j with exact domain inverses (Sec. 2.2)."""
    N = A.shape[0]
    E, O = colour_rows == 0, colour_rows == 1
    BEE = np.linalg.inv(A[np.ix_(E, E)])
    BOO = np.linalg.inv(A[np.ix_(O, O)])
    K = np.zeros((N, N), dtype=np.complex128)
    K[np.ix_(E, E)] = BEE
    K[np.ix_(O, O)] = BOO
    K[np.ix_(O, E)] = -BOO @ A[np.ix_(O, E)] @ BEE
    S = np.zeros_like(K)
    P = np.eye(N, dtype=np.complex128)
    one_minus_AK = np.eye(N) - A @ K
    for _ in range(ncycle):
        S += P
        P = P @ one_minus_AK
    return K @ S


def test_single_site_domains_closed_form(oracle_mod):
    """1^4 domains: A restricted to one site is the identity, so one MR step is
    exact (omega = 1) and K eta = (eta_E, eta_O - A_OE eta_E)."""
    dims, block = (4, 2, 2, 4), (1, 1, 1, 1)
    U = synth.su3_links(dims, 0.5, seed=51)
    eta = synth.gaussian_source(dims, 3, seed=52)
    kappa = 0.13
    col = domain_colour(dims, block)
    psi = oracle_mod.sap(dims, block, U, kappa, 1, 1, eta)
    eta_E = eta * (col == 0)[:, None, None, None]
    A_eta_E = oracle_mod.apply_D(dims, U, kappa, eta_E)
    expect = np.where((col == 0)[:, None, None, None], eta, eta - A_eta_E)
    assert np.max(np.abs(psi - expect)) < 1e-14
    # more MR steps change nothing (the domain solve is already exact)
    psi3 = oracle_mod.sap(dims, block, U, kappa, 1, 3, eta)
    assert np.max(np.abs(psi3 - expect)) < 1e-14


@pytest.mark.parametrize("ncycle", [1, 2, 3])
def test_converged_mr_equals_dense_formula(oracle_mod, small_problem, ncycle):
    dims, block, U, kappa, A = small_problem
    eta = synth.gaussian_source(dims, 2, seed=60 + ncycle)
    N = A.shape[0]
    col_rows = np.repeat(domain_colour(dims, block), 12)
    ref = _dense_sap(A, col_rows, ncycle) @ eta.reshape(N, 2)
    out = oracle_mod.sap(dims, block, U, kappa, ncycle, 60, eta).reshape(N, 2)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("mr_mode", [0, 1])
def test_one_mr_step_closed_form(oracle_mod, small_problem, mr_mode):
    """nmr = 1: on each E domain psi = omega eta with omega = (q^H eta)/(q^H q),
    q = A_dom eta; on each O domain the same on rho_O = eta_O - A_OE psi_E.
    mr_mode 0 takes one omega per column, mr_mode 1 one per domain from the
    sums over the columns."""
    dims, block, U, kappa, A = small_problem
    eta = synth.gaussian_source(dims, 2, seed=71)
    V = int(np.prod(dims))
    N = 12 * V
    col = np.repeat(domain_colour(dims, block), 12)
    dom = np.repeat(domain_index(dims, block), 12)
    e = eta.reshape(N, 2)
    psi = np.zeros_like(e)
    for c in (0, 1):
        rho = e - A @ psi
        for d in np.unique(dom[col == c]):
            rows = dom == d
            Ad = A[np.ix_(rows, rows)]
            r = rho[rows]
            q = Ad @ r
            if mr_mode == 0:
                om = np.array([np.vdot(q[:, i], r[:, i]) / np.vdot(q[:, i], q[:, i])
                               for i in range(2)])
            else:
                om = np.full(2, np.vdot(q, r) / np.vdot(q, q))
            psi[rows] = om[None, :] * r
    out = oracle_mod.sap(dims, block, U, kappa, 1, 1, eta, mr_mode=mr_mode).reshape(N, 2)
    assert np.max(np.abs(out - psi)) < 1e-13


def test_frozen_step_lengths_make_sap_linear(oracle_mod, small_problem):
    """mr_mode 2 records the block-shared step lengths into an empty (NaN)
    table and replays them afterwards.  The recording call equals mode 1, the
    replay reproduces it, and the replay is a linear operator (the stationary
    preconditioner Sec. 2.1 requires); plain MR is not linear."""
    dims, block, U, kappa, _ = small_problem
    nd = int(np.prod(dims)) // int(np.prod(block))
    ncycle, nmr = 2, 3
    table = np.full((ncycle, 2, nmr, nd), np.nan, dtype=np.complex128)
    a = synth.gaussian_source(dims, 3, seed=72)
    b = synth.gaussian_source(dims, 3, seed=73)
    rec = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, a, mr_mode=2, omega_table=table)
    assert np.max(np.abs(rec - oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, a, mr_mode=1))) < 1e-14
    # entries exist for the domains of each sweep's own colour only
    dcol = np.array([sum(np.unravel_index(d, (4 // 2,) * 4)) % 2 for d in range(nd)])
    for c in (0, 1):
        assert np.all(np.isfinite(table[:, c, :, dcol == c]))
        assert np.all(np.isnan(table[:, c, :, dcol != c]))
    rep = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, a, mr_mode=2, omega_table=table)
    assert np.max(np.abs(rep - rec)) < 1e-14 * np.max(np.abs(rec))
    M2 = lambda v: oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, v, mr_mode=2,
                                  omega_table=table)
    c1, c2 = 0.7 - 0.2j, -1.3 + 0.5j
    lin = M2(c1 * a + c2 * b) - (c1 * M2(a) + c2 * M2(b))
    assert np.max(np.abs(lin)) < 1e-13 * np.max(np.abs(rec))
    M0 = lambda v: oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, v, mr_mode=0)
    nonlin = M0(a + b) - (M0(a) + M0(b))
    assert np.max(np.abs(nonlin)) > 1e-3 * np.max(np.abs(rec))


def test_frozen_table_fills_lazily_from_a_point_source(oracle_mod):
    """A point source reaches only the domains near it in the first
    application; the other entries stay unrecorded (their residual is exactly
    zero, so their step length multiplies zero) and are recorded by a later
    application with a wider input.  The first result is unchanged when it is
    replayed with the completed table: one linear operator throughout."""
    dims, block = (8, 8, 8, 8), (2, 2, 2, 2)
    U = synth.su3_links(dims, 0.5, seed=74)
    nd = int(np.prod(dims)) // int(np.prod(block))
    ncycle, nmr, kappa = 1, 2, 0.13
    table = np.full((ncycle, 2, nmr, nd), np.nan, dtype=np.complex128)
    pt = synth.point_source(dims, 2)
    first = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, pt, mr_mode=2, omega_table=table)
    n_first = int(np.count_nonzero(np.isfinite(table)))
    assert 0 < n_first < table.size // 2
    wide = synth.gaussian_source(dims, 2, seed=75)
    oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, wide, mr_mode=2, omega_table=table)
    assert int(np.count_nonzero(np.isfinite(table))) == table.size // 2
    again = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, pt, mr_mode=2, omega_table=table)
    assert np.max(np.abs(again - first)) < 1e-14 * np.max(np.abs(first))


def test_sap_gauge_covariance(oracle_mod):
    dims, block = (4, 4, 2, 4), (2, 2, 1, 2)
    U = synth.su3_links(dims, 0.5, seed=81)
    g = synth.gauge_transform(dims, seed=82)
    eta = synth.gaussian_source(dims, 2, seed=83)
    kappa = 0.125
    lhs = oracle_mod.sap(dims, block, gauge_transform_links(dims, U, g), kappa, 2, 4,
                         gauge_transform_block(g, eta))
    rhs = gauge_transform_block(g, oracle_mod.sap(dims, block, U, kappa, 2, 4, eta))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_sap_is_homogeneous_and_columnwise(oracle_mod):
    """MR step lengths are scale invariant, so M(c eta) = c M(eta) for complex c,
    and every column is preconditioned on its own."""
    dims, block = (4, 2, 2, 4), (2, 1, 1, 2)
    U = synth.su3_links(dims, 0.5, seed=91)
    eta = synth.gaussian_source(dims, 3, seed=92)
    m = oracle_mod.sap(dims, block, U, 0.12, 2, 3, eta)
    m2 = oracle_mod.sap(dims, block, U, 0.12, 2, 3, (0.3 - 2j) * eta)
    assert np.max(np.abs(m2 - (0.3 - 2j) * m)) < 1e-13
    m1 = oracle_mod.sap(dims, block, U, 0.12, 2, 3, eta[..., 1:2])
    assert np.max(np.abs(m1[..., 0] - m[..., 1])) < 1e-15


def test_sap_rejects_odd_domain_counts(oracle_mod):
    dims = (6, 4, 4, 4)
    U = synth.su3_links(dims, 0.5, seed=1)
    eta = synth.gaussian_source(dims, 1, seed=2)
    with pytest.raises(ValueError):
        oracle_mod.sap(dims, (2, 2, 2, 2), U, 0.12, 1, 1, eta)  # 3 domains in x
