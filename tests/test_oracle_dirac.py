"""Pins for the oracle's Wilson-Dirac operator (Sec. 2.1, Eq. (hoppingterm)).

Each check comes from outside the oracle: the Clifford algebra, the free-field
momentum-space form of D, gamma5-hermiticity, gauge covariance, and the block
form of Eq. (bloclhoppingterm) (L columns = L single applications).
"""
import numpy as np
import pytest

import synth
from lattice_helpers import (CHIRAL_GAMMA, GAMMA5, coords, gauge_transform_block,
                             gauge_transform_links)


def test_gamma_clifford_algebra(oracle_mod):
    g = oracle_mod.gamma()
    I4 = np.eye(4)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0), "gamma must be Hermitian"
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2 * I4 * (mu == nu), atol=1e-15)
        # 1 -/+ gamma_mu are twice rank-2 projectors
        assert np.linalg.matrix_rank(I4 - g[mu]) == 2
        assert np.linalg.matrix_rank(I4 + g[mu]) == 2
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    assert np.allclose(g5, GAMMA5, atol=1e-15)
    # gamma_4 is not diagonal (the 1320-flop count of Sec. 2.1 needs a
    # non-diagonal gamma_4; a diagonal one gives 1296)
    assert np.count_nonzero(np.abs(np.diag(g[3]))) == 0
    assert np.allclose(g, CHIRAL_GAMMA, atol=0)


def _plane_wave(dims, n, u):
    """psi_x = exp(i p.x) u with p_mu = 2 pi n_mu / L_mu (x, y, z) and
    (2 n_t + 1) pi / L_t (antiperiodic t)."""
    p = np.array([2 * np.pi * n[0] / dims[0], 2 * np.pi * n[1] / dims[1],
                  2 * np.pi * n[2] / dims[2], (2 * n[3] + 1) * np.pi / dims[3]])
    c = coords(dims)
    ph = np.exp(1j * (c @ p))
    return ph[:, None, None, None] * u[None, :, :, :], p


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 8)])
def test_free_field_momentum_space(oracle_mod, dims):
    """U = 1: D psi = [1 - 2 kappa sum cos p_mu + 2 i kappa sum gamma_mu sin p_mu] psi
    for plane waves, and the eigenvalues of the 12x12 momentum-space matrix are
    1 - 2 kappa sum cos p +/- 2 i kappa sqrt(sum sin^2 p) (basis independent)."""
    V = int(np.prod(dims))
    U = np.tile(np.eye(3, dtype=np.complex128), (V, 4, 1, 1))
    kappa = 0.13
    rng = np.random.default_rng(5)
    for n in [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 5, 2), (2, 1, 1, 3)]:
        u = rng.standard_normal((4, 3, 3)) + 1j * rng.standard_normal((4, 3, 3))  # L = 3
        psi, p = _plane_wave(dims, n, u)
        out = oracle_mod.apply_D(dims, U, kappa, psi)
        Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
            CHIRAL_GAMMA[m] * np.sin(p[m]) for m in range(4))
        expect = np.einsum("st,vtai->vsai", Dp, psi)
        assert np.max(np.abs(out - expect)) < 1e-13
        # basis-free: the spectrum of D restricted to this momentum
        ev = np.linalg.eigvals(Dp)
        re = 1 - 2 * kappa * np.cos(p).sum()
        im = 2 * kappa * np.sqrt((np.sin(p) ** 2).sum())
        assert np.allclose(ev.real, re, atol=1e-13)
        assert np.allclose(np.sort(ev.imag), [-im, -im, im, im], atol=1e-13)


def test_gamma5_hermiticity(oracle_mod):
    """<phi, D psi> = <gamma5 D gamma5 phi, psi>, i.e. D^dagger = gamma5 D gamma5."""
    dims = (4, 4, 2, 6)
    U = synth.su3_links(dims, 0.7, seed=11)
    phi = synth.gaussian_source(dims, 2, seed=12)
    psi = synth.gaussian_source(dims, 2, seed=13)
    kappa = 0.137
    g5 = lambda v: np.einsum("st,vtai->vsai", GAMMA5, v)
    lhs = np.einsum("vsai,vsai->i", phi.conj(), oracle_mod.apply_D(dims, U, kappa, psi))
    rhs = np.einsum("vsai,vsai->i", g5(oracle_mod.apply_D(dims, U, kappa, g5(phi))).conj(), psi)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    # and it is not trivially satisfied: D itself is not Hermitian
    rhs_h = np.einsum("vsai,vsai->i", oracle_mod.apply_D(dims, U, kappa, phi).conj(), psi)
    assert np.max(np.abs(lhs - rhs_h)) > 1e-3


def test_gauge_covariance(oracle_mod):
    """D[U^g] (g psi) = g D[U] psi with U^g_mu(x) = g_x U_mu(x) g_{x+mu}^dagger."""
    dims = (4, 2, 4, 4)
    U = synth.su3_links(dims, 0.5, seed=21)
    g = synth.gauge_transform(dims, seed=22)
    psi = synth.gaussian_source(dims, 3, seed=23)
    kappa = 0.125
    lhs = oracle_mod.apply_D(dims, gauge_transform_links(dims, U, g), kappa,
                             gauge_transform_block(g, psi))
    rhs = gauge_transform_block(g, oracle_mod.apply_D(dims, U, kappa, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    # a wrong link direction convention would not be covariant: check the test bites
    U_wrong = U.copy()
    U_wrong[:, 0] = U[:, 0].conj().transpose(0, 2, 1)
    lhs_w = oracle_mod.apply_D(dims, gauge_transform_links(dims, U_wrong, g), kappa,
                               gauge_transform_block(g, psi))
    rhs_w = gauge_transform_block(g, oracle_mod.apply_D(dims, U, kappa, psi))
    assert np.max(np.abs(lhs_w - rhs_w)) > 1e-2


def test_block_equals_single_columns(oracle_mod):
    """Eq. (bloclhoppingterm): the block operator acts on each column alone."""
    dims = (2, 4, 2, 4)
    U = synth.su3_links(dims, 0.5, seed=31)
    B = synth.gaussian_source(dims, 5, seed=32)
    out = oracle_mod.apply_D(dims, U, 0.11, B)
    for i in range(5):
        one = oracle_mod.apply_D(dims, U, 0.11, B[..., i:i + 1])
        assert np.array_equal(one[..., 0], out[..., i])


def test_linearity_and_kappa_zero(oracle_mod):
    dims = (2, 2, 2, 4)
    U = synth.su3_links(dims, 0.5, seed=41)
    a = synth.gaussian_source(dims, 2, seed=42)
    b = synth.gaussian_source(dims, 2, seed=43)
    assert np.array_equal(oracle_mod.apply_D(dims, U, 0.0, a), a)
    lhs = oracle_mod.apply_D(dims, U, 0.12, (2 - 1j) * a + b)
    rhs = (2 - 1j) * oracle_mod.apply_D(dims, U, 0.12, a) + oracle_mod.apply_D(dims, U, 0.12, b)
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_antiperiodic_time_boundary(oracle_mod):
    """A source on the last time slice hops forward onto t = 0 with a factor -1
    and the forward hop carries (1 - gamma_4) U_4."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    U = np.tile(np.eye(3, dtype=np.complex128), (V, 4, 1, 1))
    psi = np.zeros((V, 4, 3, 1), dtype=np.complex128)
    s_last = 0 + 2 * (0 + 2 * (0 + 2 * 3))  # (0,0,0,3)
    psi[s_last, :, 0, 0] = [1, 2, 3, 4]
    kappa = 0.1
    out = oracle_mod.apply_D(dims, U, kappa, psi)
    g4 = CHIRAL_GAMMA[3]
    v = np.array([1, 2, 3, 4], dtype=np.complex128)
    # site (0,0,0,0): its backward t neighbour is t = 3, across the boundary, so it
    # receives -kappa * (1 + gamma_4) * (-1) * psi
    assert np.allclose(out[0, :, 0, 0], kappa * (np.eye(4) + g4) @ v, atol=1e-15)
    # site (0,0,0,2): its forward t neighbour is t = 3, no phase
    s2 = 2 * 2 * 2 * 2
    assert np.allclose(out[s2, :, 0, 0], -kappa * (np.eye(4) - g4) @ v, atol=1e-15)
    # the source site itself: diagonal term only
    assert np.allclose(out[s_last, :, 0, 0], v, atol=1e-15)
    # t = 1 is not a neighbour of t = 3 on the same (x, y, z): untouched
    assert np.max(np.abs(out[8])) == 0
