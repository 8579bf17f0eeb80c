"""The seeded synthetic inputs match the recipe stated for them: Gell-Mann
matrices normalised Tr(lambda_a lambda_b) = 2 delta_ab and closing su(3)
(traceless, Hermitian); links U = exp(i eps H) unitary with det 1 and the
eigenphases eps times those of H; Gaussian sources with Re, Im iid N(0, 1);
point sources at the given site; every generator reproducible from its seed."""
import numpy as np
import pytest

import synth


def test_gell_mann_matrices():
    lam = synth.gell_mann()
    for a in range(8):
        assert np.allclose(lam[a], lam[a].conj().T, atol=0)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2 * (a == b)) < 1e-14
    # the commutators close on the algebra: [lambda_a, lambda_b] = 2 i f_abc lambda_c
    # with real structure constants, e.g. f_123 = 1
    c = lam[0] @ lam[1] - lam[1] @ lam[0]
    assert np.allclose(c, 2j * lam[2], atol=1e-15)


@pytest.mark.parametrize("eps", [0.0, 0.4, 0.5, 2.0])
def test_links_are_su3_with_the_stated_generator(eps):
    rng = np.random.default_rng(7)
    U = synth.su3_matrices(500, eps, rng)
    I3 = np.eye(3)
    assert np.max(np.abs(U @ U.conj().transpose(0, 2, 1) - I3)) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-14
    # U = exp(i eps H): the same draw of h gives H, whose eigenvalues times eps
    # are U's eigenphases (mod 2 pi)
    rng = np.random.default_rng(7)
    h = rng.standard_normal((500, 8))
    H = np.einsum("na,aij->nij", h, synth.gell_mann() / 2)
    w = np.linalg.eigvalsh(H)
    ph = np.sort(np.angle(np.exp(1j * eps * w)), axis=1)
    uph = np.sort(np.angle(np.linalg.eigvals(U)), axis=1)
    assert np.max(np.abs(ph - uph)) < 1e-12
    if eps == 0.0:
        assert np.max(np.abs(U - I3)) < 1e-14


def test_links_layout_and_seed():
    dims = (4, 2, 2, 6)
    U = synth.su3_links(dims, 0.5, seed=11)
    assert U.shape == (96, 4, 3, 3)
    assert np.array_equal(U, synth.su3_links(dims, 0.5, seed=11))
    assert not np.allclose(U, synth.su3_links(dims, 0.5, seed=12))
    # the links are the first 4 V draws in site-major, direction-minor order
    flat = synth.su3_matrices(4 * 96, 0.5, np.random.default_rng(11))
    assert np.array_equal(U.reshape(-1, 3, 3), flat)


def test_gaussian_source_statistics():
    dims = (8, 8, 8, 8)
    B = synth.gaussian_source(dims, 4, seed=3)
    assert B.shape == (4096, 4, 3, 4) and B.dtype == np.complex128
    x = np.concatenate([B.real.ravel(), B.imag.ravel()])   # 393216 samples
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1) < 0.01
    assert abs(np.corrcoef(B.real.ravel(), B.imag.ravel())[0, 1]) < 0.01
    assert np.array_equal(B, synth.gaussian_source(dims, 4, seed=3))


def test_point_sources():
    dims = (4, 4, 4, 4)
    B = synth.point_source(dims, 12, site=5)
    flat = B.reshape(256, 12, 12)
    assert np.array_equal(flat[5], np.eye(12))
    assert not np.any(np.delete(flat, 5, axis=0))
    assert np.array_equal(synth.point_source(dims, 3, site=0).reshape(256, 12, 3)[0], np.eye(12)[:, :3])
    with pytest.raises(ValueError):
        synth.point_source(dims, 13)


def test_gauge_transform():
    g = synth.gauge_transform((2, 2, 2, 4), seed=5)
    assert g.shape == (32, 3, 3)
    assert np.max(np.abs(g @ g.conj().transpose(0, 2, 1) - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(g) - 1)) < 1e-14
