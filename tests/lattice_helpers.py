"""Test-side helpers: dense matrices built column by column from an operator,
gauge transformations, and the site/colour bookkeeping the pins need.  These
are written independently of both the oracle and the CUDA library."""
from __future__ import annotations

import numpy as np


def coords(dims):
    """Array (V, 4) of site coordinates (x, y, z, t), x fastest."""
    Lx, Ly, Lz, Lt = dims
    s = np.arange(Lx * Ly * Lz * Lt)
    return np.stack([s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)], axis=1)


def site_of(dims, c):
    Lx, Ly, Lz, Lt = dims
    c = np.asarray(c)
    return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))


def shift_site(dims, mu, step):
    """Index array: site s -> site s + step * mu (periodic)."""
    c = coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % dims[mu]
    return site_of(dims, c)


def domain_colour(dims, block):
    c = coords(dims)
    b = c // np.asarray(block)
    return (b.sum(axis=1) % 2).astype(np.int32)


def domain_index(dims, block):
    c = coords(dims)
    nb = np.asarray(dims) // np.asarray(block)
    b = c // np.asarray(block)
    return b[:, 0] + nb[0] * (b[:, 1] + nb[1] * (b[:, 2] + nb[2] * b[:, 3]))


def dense_operator(apply, dims):
    """Dense N x N matrix (N = 12 V) of a linear block operator apply(psi) that
    takes and returns (V, 4, 3, L) arrays."""
    V = int(np.prod(dims))
    N = 12 * V
    E = np.eye(N, dtype=np.complex128).reshape(V, 4, 3, N)
    return apply(E).reshape(N, N)


def gauge_transform_links(dims, U, g):
    """U^g_mu(x) = g_x U_mu(x) g_{x+mu}^dagger."""
    Ug = np.empty_like(U)
    for mu in range(4):
        fwd = shift_site(dims, mu, +1)
        Ug[:, mu] = g @ U[:, mu] @ g[fwd].conj().transpose(0, 2, 1)
    return Ug


def gauge_transform_block(g, psi):
    """(g psi)_x = g_x psi_x on the colour index, shape (V, 4, 3, L)."""
    return np.einsum("vab,vsbi->vsai", g, psi)


def rel_site_norm(a, b):
    """max over sites of |a_x - b_x| / |b_x| (norm over spin, colour, rhs)."""
    V = a.shape[0]
    d = np.linalg.norm((a - b).reshape(V, -1), axis=1)
    r = np.linalg.norm(b.reshape(V, -1), axis=1)
    return float(np.max(d / r))


CHIRAL_GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
_s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
for _k in range(3):
    CHIRAL_GAMMA[_k][:2, 2:] = -1j * _s[_k]
    CHIRAL_GAMMA[_k][2:, :2] = 1j * _s[_k]
CHIRAL_GAMMA[3][:2, 2:] = np.eye(2)
CHIRAL_GAMMA[3][2:, :2] = np.eye(2)
GAMMA5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)
