"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA library; only
the tests, the smoke check and the CPU-baseline leg of the benchmark use it.
It is independent of the CUDA path: it neither imports nor links anything from
the library package, and the library never imports it.

Array layout (numpy complex128, C-contiguous):
    links   (V, 4, 3, 3)        U[s][mu][a][b]
    block   (V, 4, 3, L)        psi[s][spin][colour][rhs]
Every function follows arXiv:1104.0737; see oracle.c for the passage each
one restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_dbl_p = ctypes.POINTER(ctypes.c_double)
_int_p = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_gamma.argtypes = [_dbl_p]
        lib.oracle_gamma.restype = None
        lib.oracle_apply_D.argtypes = [_int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p, ctypes.c_int]
        lib.oracle_domain_colour.argtypes = [_int_p, _int_p, ctypes.c_int]
        lib.oracle_sap.argtypes = [_int_p, _int_p, _dbl_p, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, _dbl_p, _dbl_p, _dbl_p,
                                   ctypes.c_int]
        lib.oracle_qr_mgs.argtypes = [_dbl_p, ctypes.c_long, ctypes.c_int, _dbl_p]
        lib.oracle_lu_solve.argtypes = [_dbl_p, _dbl_p, ctypes.c_int, ctypes.c_int]
        lib.oracle_block_bicgstab.argtypes = [
            _int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p, ctypes.c_int, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, _dbl_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            _int_p, _dbl_p, ctypes.c_int, _int_p, _dbl_p]
        lib.oracle_clover.argtypes = [_int_p, _dbl_p, ctypes.c_double, ctypes.c_double, _dbl_p]
        lib.oracle_clover_inverse.argtypes = [ctypes.c_long, _dbl_p, _dbl_p]
        lib.oracle_apply_clover_D.argtypes = [_int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p,
                                              _dbl_p, ctypes.c_int]
        lib.oracle_apply_A.argtypes = [_int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p, _dbl_p,
                                       ctypes.c_int]
        lib.oracle_ssor_domains.argtypes = [_int_p, _int_p, _dbl_p, ctypes.c_double, _dbl_p,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, _dbl_p,
                                            _dbl_p, ctypes.c_int]
        lib.oracle_sap_ext.argtypes = [_int_p, _int_p, _dbl_p, ctypes.c_double, _dbl_p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _dbl_p, ctypes.c_int, ctypes.c_double, _dbl_p, _dbl_p,
                                       ctypes.c_int]
        lib.oracle_block_bicgstab_ext.argtypes = [
            _int_p, _dbl_p, ctypes.c_double, _dbl_p, _dbl_p, _dbl_p, ctypes.c_int,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, _dbl_p, ctypes.c_int, ctypes.c_int,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _int_p, _dbl_p,
            ctypes.c_int, _int_p, _dbl_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(_dbl_p) if a is not None else None


def _ivec(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _cplx(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def num_threads() -> int:
    return _load().oracle_num_threads()


def gamma() -> np.ndarray:
    """gamma_1..gamma_4 of the chiral basis, shape (4, 4, 4)."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    _load().oracle_gamma(_dp(g))
    return g


def domain_colour(dims, block) -> np.ndarray:
    """Colour (0 = E, 1 = O) of the SAP domain of every site."""
    lib = _load()
    V = int(np.prod(dims))
    d, b = _ivec(dims), _ivec(block)
    return np.array([lib.oracle_domain_colour(d, b, s) for s in range(V)], dtype=np.int32)


def apply_D(dims, U, kappa: float, psi) -> np.ndarray:
    """A psi for the Wilson-Dirac matrix A (Sec. 2.1), column by column."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    psi = _cplx(psi)
    if psi.ndim != 4 or psi.shape[:3] != (V, 4, 3):
        raise ValueError("psi must have shape (V, 4, 3, L)")
    out = np.empty_like(psi)
    rc = _load().oracle_apply_D(_ivec(dims), _dp(U), float(kappa), _dp(psi), _dp(out), psi.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_apply_D returned {rc}")
    return out


MR_COLUMN, MR_BLOCK, MR_FROZEN = 0, 1, 2
DOMAIN_MR, DOMAIN_SSOR = 0, 1      # SAP domain solvers (sap_ext, block_bicgstab)


def sap(dims, block, U, kappa: float, ncycle: int, nmr: int, eta, mr_mode: int = MR_COLUMN,
        omega_table=None) -> np.ndarray:
    """psi = M_SAP eta (Sec. 2.2) with nmr-step MR domain solves.

    mr_mode 0: step lengths per domain and column; 1: per domain, shared by the
    columns; 2: frozen in omega_table (NaN entries are recorded from the
    mode-1 sums the first time their domain's residual is nonzero).
    omega_table: complex array (ncycle, 2, nmr, n_domains)."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    eta = _cplx(eta)
    out = np.empty_like(eta)
    if omega_table is not None:
        nd = V // int(np.prod(block))
        if (omega_table.dtype != np.complex128 or not omega_table.flags.c_contiguous
                or omega_table.shape != (ncycle, 2, nmr, nd)):
            raise ValueError("omega_table must be a C-contiguous complex128 (ncycle, 2, nmr, nd) array")
    rc = _load().oracle_sap(_ivec(dims), _ivec(block), _dp(U), float(kappa), int(ncycle),
                            int(nmr), int(mr_mode), _dp(omega_table), _dp(eta), _dp(out),
                            eta.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_sap returned {rc}")
    return out


def qr_mgs(P):
    """P = Q gamma by modified Gram-Schmidt.  P: (N, L).  Returns (Q, gamma)."""
    Q = _cplx(P).copy()
    N, L = Q.shape
    g = np.zeros((L, L), dtype=np.complex128)
    rc = _load().oracle_qr_mgs(_dp(Q), N, L, _dp(g))
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle_qr_mgs returned {rc}")
    return Q, g


def lu_solve(G, C) -> np.ndarray:
    """Solve G X = C by LU with partial pivoting.  G: (L, L), C: (L, M)."""
    G = _cplx(G)
    X = _cplx(C).copy()
    rc = _load().oracle_lu_solve(_dp(G), _dp(X), G.shape[0], X.shape[1])
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle_lu_solve returned {rc}")
    return X


def block_bicgstab(dims, U, kappa: float, B, tol: float, max_iter: int = 1000, X0=None,
                   rtilde=None, ncycle: int = 0, nmr: int = 0, block=None,
                   mr_mode: int = MR_COLUMN, history_len: int | None = None, Tinv=None,
                   solver: int = DOMAIN_MR, nssor: int = 1, omega: float = 1.26) -> dict:
    """Algorithm 1 of Sec. 2.1 for A X = B.  A is the Wilson matrix, or with
    Tinv the Jacobi-preconditioned clover matrix T^{-1} D_c (Sec. 2.2; pass
    T^{-1} B to solve D_c X = B).  The SAP domain solver is MR (nmr, mr_mode)
    or SSOR (nssor, omega).  Returns dict(X, iters, status, history, true_res)."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    B = _cplx(B)
    L = B.shape[3]
    X = np.zeros_like(B) if X0 is None else _cplx(X0).copy()
    rt = None if rtilde is None else _cplx(rtilde, B.shape)
    Ti = None if Tinv is None else _cplx(Tinv, (V, 12, 12))
    hl = max_iter if history_len is None else history_len
    hist = np.zeros(max(hl, 1))
    iters = ctypes.c_int(0)
    tres = np.zeros(L)
    blk = _ivec(block if block is not None else (1, 1, 1, 1))
    rc = _load().oracle_block_bicgstab_ext(
        _ivec(dims), _dp(U), float(kappa), _dp(Ti), _dp(B), _dp(X), L, float(tol),
        int(max_iter), int(X0 is not None), _dp(rt), int(ncycle), int(solver), int(nmr),
        int(mr_mode), int(nssor), float(omega), blk, _dp(hist), hl, ctypes.byref(iters),
        _dp(tres))
    if rc < 0:
        raise ValueError(f"oracle_block_bicgstab_ext returned {rc}")
    k = iters.value
    return dict(X=X, iters=k, status=rc, history=hist[:min(k, hl)].copy(), true_res=tres)


# ---------------------------------------------------------------------------
# Sec. 2.2: clover term, Jacobi preconditioning, SSOR domain solves
# ---------------------------------------------------------------------------


def clover(dims, U, kappa: float, csw: float) -> np.ndarray:
    """T_x = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x), shape (V, 12, 12)
    (index spin * 3 + colour); F from the four-plaquette clover leaf."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    T = np.empty((V, 12, 12), dtype=np.complex128)
    rc = _load().oracle_clover(_ivec(dims), _dp(U), float(kappa), float(csw), _dp(T))
    if rc != 0:
        raise ValueError(f"oracle_clover returned {rc}")
    return T


def clover_inverse(T) -> np.ndarray:
    """T_x^{-1} at every site."""
    T = _cplx(T)
    if T.ndim != 3 or T.shape[1:] != (12, 12):
        raise ValueError("T must have shape (V, 12, 12)")
    Ti = np.empty_like(T)
    rc = _load().oracle_clover_inverse(T.shape[0], _dp(T), _dp(Ti))
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle_clover_inverse returned {rc}")
    return Ti


def _block_arg(dims, psi):
    V = int(np.prod(dims))
    psi = _cplx(psi)
    if psi.ndim != 4 or psi.shape[:3] != (V, 4, 3):
        raise ValueError("psi must have shape (V, 4, 3, L)")
    return psi


def apply_clover_D(dims, U, kappa: float, T, psi) -> np.ndarray:
    """D_c psi = T psi - kappa H psi."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    T = _cplx(T, (V, 12, 12))
    psi = _block_arg(dims, psi)
    out = np.empty_like(psi)
    rc = _load().oracle_apply_clover_D(_ivec(dims), _dp(U), float(kappa), _dp(T), _dp(psi),
                                       _dp(out), psi.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_apply_clover_D returned {rc}")
    return out


def apply_A(dims, U, kappa: float, Tinv, psi) -> np.ndarray:
    """A psi, A = T^{-1} D_c = 1 - kappa T^{-1} H (Wilson D when Tinv is None)."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    Ti = None if Tinv is None else _cplx(Tinv, (V, 12, 12))
    psi = _block_arg(dims, psi)
    out = np.empty_like(psi)
    rc = _load().oracle_apply_A(_ivec(dims), _dp(U), float(kappa), _dp(Ti), _dp(psi), _dp(out),
                                psi.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_apply_A returned {rc}")
    return out


def ssor_domains(dims, block, U, kappa: float, nssor: int, omega: float, colour: int, psi,
                 Tinv=None) -> np.ndarray:
    """B_cc psi: the SSOR domain solve of Sec. 2.2 on every domain of one colour."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    Ti = None if Tinv is None else _cplx(Tinv, (V, 12, 12))
    psi = _block_arg(dims, psi)
    out = np.empty_like(psi)
    rc = _load().oracle_ssor_domains(_ivec(dims), _ivec(block), _dp(U), float(kappa), _dp(Ti),
                                     int(nssor), float(omega), int(colour), _dp(psi), _dp(out),
                                     psi.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_ssor_domains returned {rc}")
    return out


def sap_ext(dims, block, U, kappa: float, ncycle: int, eta, Tinv=None, solver: int = DOMAIN_SSOR,
            nmr: int = 0, mr_mode: int = MR_COLUMN, omega_table=None, nssor: int = 1,
            omega: float = 1.26) -> np.ndarray:
    """psi = M_SAP eta (Sec. 2.2) for the matrix of apply_A, with MR or SSOR
    domain solves."""
    V = int(np.prod(dims))
    U = _cplx(U, (V, 4, 3, 3))
    Ti = None if Tinv is None else _cplx(Tinv, (V, 12, 12))
    eta = _block_arg(dims, eta)
    out = np.empty_like(eta)
    if omega_table is not None:
        nd = V // int(np.prod(block))
        if (omega_table.dtype != np.complex128 or not omega_table.flags.c_contiguous
                or omega_table.shape != (ncycle, 2, nmr, nd)):
            raise ValueError("omega_table must be a C-contiguous complex128 (ncycle, 2, nmr, nd) array")
    rc = _load().oracle_sap_ext(_ivec(dims), _ivec(block), _dp(U), float(kappa), _dp(Ti),
                                int(ncycle), int(solver), int(nmr), int(mr_mode), _dp(omega_table),
                                int(nssor), float(omega), _dp(eta), _dp(out), eta.shape[3])
    if rc != 0:
        raise ValueError(f"oracle_sap_ext returned {rc}")
    return out


# ---------------------------------------------------------------------------
# FP16 storage format (numpy; no arithmetic of the method, only rounding)
# ---------------------------------------------------------------------------
def quantize_fp16(psi) -> np.ndarray:
    """The block that FP16 storage with one scale per (site, rhs) represents.

    For every site and column the scale is the largest |re| or |im| of the
    spinor (12 complex numbers), rounded to FP32; each real component divided
    by it (in FP64) is rounded to nearest FP16; the value represented is the
    FP16 number times the scale, exactly.  A zero spinor stays zero.
    psi: (V, 4, 3, L) complex128."""
    psi = np.asarray(psi, dtype=np.complex128)
    V, L = psi.shape[0], psi.shape[-1]
    parts = np.stack([psi.real, psi.imag], axis=-1).reshape(V, 12, L, 2)
    m = np.abs(parts).max(axis=(1, 3))                      # (V, L)
    s = m.astype(np.float32).astype(np.float64)
    safe = np.where(s > 0, s, 1.0)
    q = (parts / safe[:, None, :, None]).astype(np.float16).astype(np.float64)
    out = q * s[:, None, :, None]
    return (out[..., 0] + 1j * out[..., 1]).reshape(psi.shape)


def quantize_links_fp16(U) -> np.ndarray:
    """Links as FP16 storage of their first two rows represents them: rows 0
    and 1 rounded component-wise to FP16 (no scale: |U_ab| <= 1), row 2 rebuilt
    as the complex conjugate of the cross product of rows 0 and 1 (the
    relation that holds for SU(3)).  U: (V, 4, 3, 3) complex128."""
    U = np.asarray(U, dtype=np.complex128)
    r = U[..., :2, :]
    rq = r.real.astype(np.float16).astype(np.float64) + 1j * r.imag.astype(np.float16).astype(np.float64)
    row2 = np.conj(np.cross(rq[..., 0, :], rq[..., 1, :]))
    return np.concatenate([rq, row2[..., None, :]], axis=-2)
