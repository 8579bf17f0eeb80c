"""Seeded synthetic inputs shared by the oracle checks, the CUDA parity tests
and the benchmark.

This module holds input generation only (gauge links, sources, random gauge
transformations); none of the solver's arithmetic lives here.  Arrays use the
library's external layout:

    links   U[s][mu][a][b]          complex128, shape (V, 4, 3, 3)
    block   psi[s][spin][colour][i] complex128, shape (V, 4, 3, L)

with s = x + Lx*(y + Ly*(z + Lz*t)) and mu = 0..3 for x, y, z, t.

The paper's PACS-CS gauge configurations (Sec. 3.1) are not available; the
links here are independent SU(3) matrices U = exp(i eps H), H = sum_a h_a
lambda_a / 2 with Gell-Mann matrices lambda_a and h_a ~ N(0, 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume",
    "gell_mann",
    "su3_matrices",
    "su3_links",
    "gaussian_source",
    "point_source",
    "gauge_transform",
]


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def su3_matrices(n: int, eps: float, rng: np.random.Generator, chunk: int = 1 << 20) -> np.ndarray:
    """n matrices exp(i eps H) with H = sum_a h_a lambda_a / 2, h_a ~ N(0,1)."""
    lam = gell_mann() / 2
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for k0 in range(0, n, chunk):
        k1 = min(n, k0 + chunk)
        h = rng.standard_normal((k1 - k0, 8))
        H = np.einsum("na,aij->nij", h, lam)
        w, vec = np.linalg.eigh(H)
        ph = np.exp(1j * eps * w)
        out[k0:k1] = np.einsum("nij,nj,nkj->nik", vec, ph, vec.conj())
    return out


def su3_links(dims, eps: float, seed: int) -> np.ndarray:
    """Seeded gauge field, shape (V, 4, 3, 3)."""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    return su3_matrices(4 * V, eps, rng).reshape(V, 4, 3, 3)


def gaussian_source(dims, L: int, seed: int) -> np.ndarray:
    """Block of L complex Gaussian vectors (Re, Im iid N(0,1)), shape (V, 4, 3, L)."""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    re = rng.standard_normal((V, 4, 3, L))
    im = rng.standard_normal((V, 4, 3, L))
    return re + 1j * im


def point_source(dims, L: int = 12, site: int = 0) -> np.ndarray:
    """Local sources of Sec. 3.1: column i is the unit vector at `site` with
    spin*3 + colour = i (i < 12)."""
    if not 1 <= L <= 12:
        raise ValueError("point sources exist for 1 <= L <= 12")
    V = volume(dims)
    b = np.zeros((V, 12, L), dtype=np.complex128)
    for i in range(L):
        b[site, i, i] = 1.0
    return b.reshape(V, 4, 3, L)


def gauge_transform(dims, seed: int, eps: float = 2.0) -> np.ndarray:
    """One seeded SU(3) matrix per site, shape (V, 3, 3)."""
    rng = np.random.default_rng(seed)
    return su3_matrices(volume(dims), eps, rng)
