"""The block linear algebra kernels of the CUDA path, compiled for the host and
run with one host thread per CUDA thread (tests/host_emulation/
shim_threads.h; the Gram kernel's bulk copies and mbarrier waits emulated),
against their plain definitions: the fused block inner products of Algorithm 2
(R~^H V with R~^H R; R~^H Z with Tr(Z^H R) and Tr(Z^H Z); the P^H P of the QR;
FP64 and FP32 storage, ragged last tile, several CTAs), the block updates
(R -= V alpha; X += U alpha + zeta S, R -= zeta Z and P = R + (P - zeta V) beta
with the column norms; Y = X M of the QR), the one-CTA L x L kernels: LU with partial
pivoting for alpha and beta, zeta, and the Cholesky factor's inverse (plain
and shifted) of CholeskyQR; and the conversions: ABI <-> internal layout,
the link copies with their NaN and SU(3) checks, the residual B - W with its
column norms, the input scan, and the dummy right-hand-side columns."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import emulation_sources

HERE = os.path.join(emulation_sources.ROOT, "tests", "host_emulation")
CUDA_INCLUDE = "/usr/local/cuda/include"
ST_ALPHA_SINGULAR, ST_ZZ_ZERO, ST_CHOL_FAIL = 1, 2, 4


@pytest.fixture(scope="module")
def blas(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INCLUDE, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("blas_emulation")
    (d / "blas_parts.inc").write_text(emulation_sources.blas_parts())
    shutil.copy(os.path.join(HERE, "shim_threads.h"), d / "shim_threads.h")
    lib_path = d / "libblas.so"
    subprocess.run(["g++", "-std=c++20", "-O1", "-fPIC", "-shared", "-pthread", "-I", str(d), "-I", CUDA_INCLUDE,
                    os.path.join(HERE, "blas_harness.cpp"), "-o", str(lib_path)], check=True)
    lib = ctypes.CDLL(str(lib_path))
    D, I, V = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
    lib.emu_lxl_alpha.argtypes = [ctypes.c_int, D, ctypes.c_int, D, D, I, D]
    lib.emu_lxl_zeta_beta.argtypes = [ctypes.c_int, D, ctypes.c_int, D, I, D, ctypes.c_int]
    lib.emu_lxl_chol.argtypes = [ctypes.c_int, D, ctypes.c_int, D, ctypes.c_double, ctypes.c_double]
    lib.emu_gram.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, V, V, V, ctypes.c_int, D]
    lib.emu_convert.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, V, V]
    lib.emu_convert_links.argtypes = [ctypes.c_longlong, D, D, ctypes.POINTER(ctypes.c_float)]
    lib.emu_residual_from.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, D, D, V, D, ctypes.c_int]
    lib.emu_abi_check.argtypes = [ctypes.c_longlong, ctypes.c_int, D, D, ctypes.c_int]
    lib.emu_pack_dummies.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, D, D, ctypes.c_ulonglong,
                                     ctypes.c_int]
    lib.emu_first_columns.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_int, D, D]
    lib.emu_updates.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, V, D, V, V, V,
                                D, V, V, V, D, D, V]
    return lib


def _d(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _v(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _mat(blk):
    """Internal block [site][rhs][12] -> matrix with rows (site, spin-colour), columns rhs."""
    return blk.transpose(0, 2, 1).reshape(-1, blk.shape[1])


def _partials(rng, slots, nparts):
    """nparts partial sums (nparts, nslots, 2) whose sum is `slots` (complex)."""
    parts = _rand(rng, nparts, slots.size) * 0.1
    parts[-1] = slots - parts[:-1].sum(0)
    return np.ascontiguousarray(np.stack([parts.real, parts.imag], -1))


def _slots(L, G1=None, G2=None, D1=None, D2=None):
    s = np.zeros(2 * L * L + 2 * L, complex)
    if G1 is not None:
        s[:L * L] = G1.ravel()
    if G2 is not None:
        s[L * L:2 * L * L] = G2.ravel()
    if D1 is not None:
        s[2 * L * L:2 * L * L + L] = D1
    if D2 is not None:
        s[2 * L * L + L:] = D2
    return s


# ---------------------------------------------------------------------------
# L x L kernels
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L", [1, 4, 12, 16])
def test_alpha_and_beta_solves(blas, L):
    rng = np.random.default_rng(L)
    G = _rand(rng, L, L)
    if L > 1:
        G[0, 0] = 0  # the first column needs a row interchange
    C = _rand(rng, L, L)
    part = _partials(rng, _slots(L, G, C), 3)
    Gout, LU, alpha = (np.zeros(2 * L * L) for _ in range(3))
    piv = np.zeros(L, np.int32)
    st = blas.emu_lxl_alpha(L, _d(part), 3, _d(Gout), _d(LU), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _d(alpha))
    assert st == 0
    a = (alpha[0::2] + 1j * alpha[1::2]).reshape(L, L)
    ref = np.linalg.solve(G, C)
    assert np.max(np.abs(a - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.allclose((Gout[0::2] + 1j * Gout[1::2]).reshape(L, L), G, rtol=0, atol=1e-13)
    # beta = -G^{-1} (R~^H Z) with the same factors; zeta = sum D1 / sum Re D2
    RZ = _rand(rng, L, L)
    D1 = _rand(rng, L)
    D2 = np.abs(_rand(rng, L)) ** 2
    part2 = _partials(rng, _slots(L, RZ, None, D1, D2), 2)
    zb = np.zeros(2 + 2 * L * L)
    st = blas.emu_lxl_zeta_beta(L, _d(part2), 2, _d(LU), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(zb), 0)
    assert st == 0
    zeta = zb[0] + 1j * zb[1]
    assert abs(zeta - D1.sum() / D2.sum()) < 1e-13 * abs(zeta)
    beta = (zb[2::2] + 1j * zb[3::2]).reshape(L, L)
    ref = -np.linalg.solve(G, RZ)
    assert np.max(np.abs(beta - ref)) < 1e-12 * np.max(np.abs(ref))


def test_lxl_statuses(blas):
    L = 4
    rng = np.random.default_rng(7)
    G = _rand(rng, L, L)
    G[:, 2] = G[:, 1]  # singular
    part = _partials(rng, _slots(L, G, _rand(rng, L, L)), 1)
    buf = [np.zeros(2 * L * L) for _ in range(3)]
    piv = np.zeros(L, np.int32)
    st = blas.emu_lxl_alpha(L, _d(part), 1, _d(buf[0]), _d(buf[1]), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            _d(buf[2]))
    assert st & ST_ALPHA_SINGULAR and not np.any(buf[2])
    zb = np.zeros(2 + 2 * L * L)
    part2 = _partials(rng, _slots(L, _rand(rng, L, L), None, _rand(rng, L), np.zeros(L)), 1)
    st = blas.emu_lxl_zeta_beta(L, _d(part2), 1, _d(buf[1]), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                _d(zb), 0)
    assert st & ST_ZZ_ZERO and not np.any(zb)


@pytest.mark.parametrize("L", [1, 5, 12])
@pytest.mark.parametrize("shift", [0.0, 1e-5])
def test_cholesky_inverse(blas, L, shift):
    rng = np.random.default_rng(10 + L)
    P = _rand(rng, 200, L)
    G = P.conj().T @ P
    part = _partials(rng, _slots(L, G), 4)
    M = np.zeros(2 * L * L)
    st = blas.emu_lxl_chol(L, _d(part), 4, _d(M), 1e-26, shift)
    assert st == 0
    Mc = (M[0::2] + 1j * M[1::2]).reshape(L, L)
    Gs = G + shift * np.max(np.diag(G).real) * np.eye(L)
    gamma = np.linalg.cholesky(Gs).conj().T  # upper triangular, real positive diagonal
    assert np.max(np.abs(Mc - np.linalg.inv(gamma))) < 1e-12 * np.max(np.abs(Mc))
    assert np.allclose(np.tril(Mc, -1), 0, atol=0)


def test_cholesky_failure(blas):
    L = 4
    rng = np.random.default_rng(3)
    P = _rand(rng, 50, L)
    P[:, 3] = P[:, 0]  # rank deficient
    part = _partials(rng, _slots(L, P.conj().T @ P), 1)
    M = np.zeros(2 * L * L)
    st = blas.emu_lxl_chol(L, _d(part), 1, _d(M), 1e-26, 0.0)
    assert st & ST_CHOL_FAIL
    # the failed factor leaves the identity, so the block is not changed
    assert np.allclose((M[0::2] + 1j * M[1::2]).reshape(L, L), np.eye(L), atol=0)


# ---------------------------------------------------------------------------
# Gram kernel
# ---------------------------------------------------------------------------
GRAM_CASES = [  # (flags, A is B1)
    (1 | 2, False),       # R~^H V and R~^H R (the alpha system)
    (1, True),            # P^H P of the QR (Hermitian path)
    (1 | 4 | 8, False),   # R~^H Z, diag(Z^H R), diag(Z^H Z) (zeta and the beta system)
]


@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("L", [3, 4, 5, 12])
@pytest.mark.parametrize("flags,herm", GRAM_CASES)
def test_gram_kernel(blas, fp64, L, flags, herm):
    rng = np.random.default_rng(100 * L + flags)
    nsite = 101  # a ragged last tile
    dt = np.complex128 if fp64 else np.complex64
    A, B1, B2 = (np.ascontiguousarray(_rand(rng, nsite, L, 12).astype(dt)) for _ in range(3))
    if herm:
        A = B1
    nslots = 2 * L * L + 2 * L
    part = np.zeros((400, nslots, 2))
    n = blas.emu_gram(fp64, L, nsite, _v(A), _v(B1), _v(B2) if flags & 2 or flags & 4 else None, flags, _d(part))
    assert n > 1
    tot = part[:n, :, 0].sum(0) + 1j * part[:n, :, 1].sum(0)
    a, b1, b2 = (_mat(x.astype(np.complex128)) for x in (A, B1, B2))
    _check_gram(tot, L, flags, a, b1, b2, nsite, fp64)


def _check_gram(tot, L, flags, a, b1, b2, nsite, fp64):
    """Each requested product within the rounding of its sum: relative to the
    size of the terms (|x||y| summed over the 12 nsite rows)."""
    u = 1e-15 if fp64 else 1e-7
    n = nsite * 12

    def close(got, ref, terms):
        assert np.all(np.abs(got - ref) < 40 * u * np.sqrt(n) * terms)

    if flags & 1:
        close(tot[:L * L].reshape(L, L), a.conj().T @ b1, np.abs(a).T @ np.abs(b1))
    if flags & 2:
        close(tot[L * L:2 * L * L].reshape(L, L), a.conj().T @ b2, np.abs(a).T @ np.abs(b2))
    if flags & 4:
        close(tot[2 * L * L:2 * L * L + L], np.sum(b1.conj() * b2, 0), np.sum(np.abs(b1) * np.abs(b2), 0))
    if flags & 8:
        close(tot[2 * L * L + L:], np.sum(np.abs(b1) ** 2, 0), np.sum(np.abs(b1) ** 2, 0))


@pytest.mark.parametrize("fp64", [1, 0])
def test_gram_kernel_pipeline(blas, fp64):
    """More tiles than CTAs: every CTA walks several tiles through the two
    shared-memory stages, re-arming each mbarrier for the next phase."""
    L, flags = 4, 1 | 2 | 4 | 8
    rng = np.random.default_rng(300 + fp64)
    ts = 8 if fp64 else 16                 # sites per tile
    nsite = 304 * ts * 3 + 5               # three tiles and more for each of the 304 CTAs
    dt = np.complex128 if fp64 else np.complex64
    A, B1, B2 = (np.ascontiguousarray(_rand(rng, nsite, L, 12).astype(dt)) for _ in range(3))
    nslots = 2 * L * L + 2 * L
    part = np.zeros((400, nslots, 2))
    n = blas.emu_gram(fp64, L, nsite, _v(A), _v(B1), _v(B2), flags, _d(part))
    assert n == 304
    tot = part[:n, :, 0].sum(0) + 1j * part[:n, :, 1].sum(0)
    a, b1, b2 = (_mat(x.astype(np.complex128)) for x in (A, B1, B2))
    _check_gram(tot, L, flags, a, b1, b2, nsite, fp64)


# ---------------------------------------------------------------------------
# block updates
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("L", [3, 12])
def test_block_updates(blas, fp64, L):
    rng = np.random.default_rng(200 + L)
    nsite, ncta = 37, 3
    nrow = nsite * 12
    dt = np.complex128 if fp64 else np.complex64
    tol = 1e-13 if fp64 else 1e-5
    U, S, Z, V, R, P = (np.ascontiguousarray(_rand(rng, nsite, L, 12).astype(dt)) for _ in range(6))
    X0 = np.ascontiguousarray(_rand(rng, nsite, L, 12))
    alpha, beta, M = _rand(rng, L, L), _rand(rng, L, L), _rand(rng, L, L)
    zeta = 0.3 - 0.7j
    pack = lambda m: np.ascontiguousarray(np.stack([m.real, m.imag], -1).ravel())
    zb = np.concatenate([[zeta.real, zeta.imag], pack(beta)])
    m = lambda x: _mat(x.astype(np.complex128))
    scale = lambda ref: tol * max(1.0, np.max(np.abs(ref)))
    # Y = X M
    Y = np.zeros_like(U)
    blas.emu_updates(fp64, L, 0, ncta, nrow, _v(U), None, None, None, None, None, None, None, None, None, _d(pack(M)),
                     _v(Y))
    ref = m(U) @ M
    assert np.max(np.abs(m(Y) - ref)) < scale(ref)
    # R -= V alpha
    R1 = R.copy()
    blas.emu_updates(fp64, L, 1, ncta, nrow, None, _d(pack(alpha)), None, None, _v(V), None, _v(R1), None, None, None,
                     None, None)
    ref = m(R) - m(V) @ alpha
    assert np.max(np.abs(m(R1) - ref)) < scale(ref)
    # X += U alpha + zeta S, R -= zeta Z, P = R + (P - zeta V) beta, column norms of the new R
    R2, P2, X2 = R.copy(), P.copy(), X0.copy()
    part = np.zeros((ncta, L))
    blas.emu_updates(fp64, L, 2, ncta, nrow, _v(U), _d(pack(alpha)), _v(S), _v(Z), _v(V), _d(zb), _v(R2), _v(P2),
                     _v(X2), _d(part), None, None)
    xr = _mat(X0) + m(U) @ alpha + zeta * m(S)
    rr = m(R) - zeta * m(Z)
    pr = rr + (m(P) - zeta * m(V)) @ beta
    # X accumulates in FP64: only the increment carries the vectors' rounding
    assert np.max(np.abs(_mat(X2) - xr)) < tol * max(1.0, np.max(np.abs(xr - _mat(X0))))
    assert np.max(np.abs(m(R2) - rr)) < scale(rr)
    assert np.max(np.abs(m(P2) - pr)) < scale(pr)
    assert np.max(np.abs(part.sum(0) - np.sum(np.abs(m(R2)) ** 2, 0))) < tol * np.max(np.sum(np.abs(rr) ** 2, 0))


# ---------------------------------------------------------------------------
# conversions, input checks, dummy columns
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fp64", [1, 0])
def test_layout_conversions(blas, fp64):
    rng = np.random.default_rng(400)
    nsite, L = 53, 5
    abi = np.ascontiguousarray(_rand(rng, nsite, 12, L))        # [site][spin*3+colour][rhs]
    dt = np.complex128 if fp64 else np.complex64
    internal = np.zeros((nsite, L, 12), dt)
    blas.emu_convert(fp64, 1, nsite, L, _v(abi), _v(internal))
    assert np.array_equal(internal, abi.transpose(0, 2, 1).astype(dt))
    back = np.zeros_like(abi)
    blas.emu_convert(fp64, 0, nsite, L, _v(internal), _v(back))
    assert np.array_equal(back, abi.astype(dt).astype(np.complex128))


def _su3(rng, n):
    H = _rand(rng, n, 3, 3)
    H = (H + H.conj().transpose(0, 2, 1)) / 2
    H -= np.trace(H, axis1=1, axis2=2)[:, None, None] * np.eye(3) / 3
    w, v = np.linalg.eigh(H)
    return v @ (np.exp(0.5j * w)[..., None] * v.conj().transpose(0, 2, 1))


def test_link_conversion_and_checks(blas):
    rng = np.random.default_rng(401)
    n = 300
    U = np.ascontiguousarray(_su3(rng, n))
    l64, l32 = np.zeros_like(U), np.zeros(U.shape, np.complex64)
    f32 = ctypes.POINTER(ctypes.c_float)
    assert blas.emu_convert_links(n, _d(U), _d(l64), l32.ctypes.data_as(f32)) == 0
    assert np.array_equal(l64, U) and np.array_equal(l32, U.astype(np.complex64))
    bad = U.copy()
    bad[7] *= np.exp(0.1j)  # unitary, det != 1
    assert blas.emu_convert_links(n, _d(bad), _d(l64), l32.ctypes.data_as(f32)) == 2
    bad = U.copy()
    bad[9, 1, 2] += 1e-8  # not unitary
    assert blas.emu_convert_links(n, _d(bad), _d(l64), l32.ctypes.data_as(f32)) == 2
    bad = U.copy()
    bad[11, 0, 0] = np.nan
    assert blas.emu_convert_links(n, _d(bad), _d(l64), l32.ctypes.data_as(f32)) & 1


@pytest.mark.parametrize("fp64", [1, 0])
@pytest.mark.parametrize("L", [1, 5, 12])
def test_residual_and_input_scan(blas, fp64, L):
    rng = np.random.default_rng(402 + L)
    nsite, ncta = 41, 3
    B, W = (np.ascontiguousarray(_rand(rng, nsite, L, 12)) for _ in range(2))
    dt = np.complex128 if fp64 else np.complex64
    out = np.zeros((nsite, L, 12), dt)
    part = np.zeros((ncta, L))
    blas.emu_residual_from(fp64, nsite, L, _d(B), _d(W), _v(out), _d(part), ncta)
    r = B - W
    assert np.array_equal(out, r.astype(dt))
    assert np.allclose(part.sum(0), np.sum(np.abs(r) ** 2, axis=(0, 2)), rtol=1e-14, atol=0)
    blas.emu_residual_from(fp64, nsite, L, _d(B), None, _v(out), _d(part), ncta)  # W = NULL: R = B
    assert np.array_equal(out, B.astype(dt))
    # the ABI input scan: column norms and NaN/Inf
    abi = np.ascontiguousarray(_rand(rng, nsite * 12, L))
    part = np.zeros((ncta, L))
    assert blas.emu_abi_check(nsite * 12, L, _d(abi), _d(part), ncta) == 0
    assert np.allclose(part.sum(0), np.sum(np.abs(abi) ** 2, 0), rtol=1e-14, atol=0)
    abi[17, L - 1] = np.inf
    assert blas.emu_abi_check(nsite * 12, L, _d(abi), _d(part), ncta) & 1


def test_dummy_columns(blas):
    """The first L columns copied, the others seeded Gaussian numbers (zeros
    when not random), the same for the same seed; first_columns inverts it."""
    rng = np.random.default_rng(403)
    nrow, L, Lt = 12 * 500, 3, 8
    B = np.ascontiguousarray(_rand(rng, nrow, L))
    out, out2, zero = (np.zeros((nrow, Lt), complex) for _ in range(3))
    blas.emu_pack_dummies(nrow, L, Lt, _d(B), _d(out), 12345, 1)
    blas.emu_pack_dummies(nrow, L, Lt, _d(B), _d(out2), 12345, 1)
    blas.emu_pack_dummies(nrow, L, Lt, _d(B), _d(zero), 12345, 0)
    assert np.array_equal(out[:, :L], B) and np.array_equal(out, out2)
    assert not np.any(zero[:, L:])
    d = out[:, L:].ravel()
    x = np.concatenate([d.real, d.imag])
    assert abs(x.mean()) < 0.02 and abs(x.var() - 1.0) < 0.03     # N(0, 1) parts, 60000 samples
    assert abs(np.corrcoef(d.real, d.imag)[0, 1]) < 0.02
    other = np.zeros_like(out)
    blas.emu_pack_dummies(nrow, L, Lt, _d(B), _d(other), 54321, 1)
    assert not np.allclose(other[:, L:], out[:, L:])
    first = np.zeros((nrow, L), complex)
    blas.emu_first_columns(nrow, Lt, L, _d(out), _d(first))
    assert np.array_equal(first, B)
