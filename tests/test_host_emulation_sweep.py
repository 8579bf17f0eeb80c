"""The fused SAP sweep kernel (Sec. 2.2) of the CUDA path, compiled for the
host and run with one host thread per CUDA thread (tests/host_emulation/
shim_threads.h: real barriers for __syncthreads, the cluster barrier and warp
shuffles; one shared-memory arena per CTA, read across the cluster through
emulated distributed shared memory), against the oracle's SAP in FP32
tolerance: the 4^4 variant (one CTA per domain) and the 8^4 variant (an
8-CTA cluster per domain), per-column MR and frozen step lengths, several
persistent clusters sharing the (domain, column) items unevenly.

This checks the sweep's index maps, its on-chip data flow and its barriers'
placement for reads of data no thread has written (shared memory starts as
NaN) on a machine without a GPU; timing and the real memory model are left
to the -m gpu tests."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import emulation_sources
import synth

HERE = os.path.join(emulation_sources.ROOT, "tests", "host_emulation")
CUDA_INCLUDE = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def sweep(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INCLUDE, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("sweep_emulation")
    (d / "sweep_parts.inc").write_text(emulation_sources.sweep_parts())
    shutil.copy(os.path.join(HERE, "shim_threads.h"), d / "shim_threads.h")
    lib_path = d / "libsweep.so"
    subprocess.run(["g++", "-std=c++20", "-O2", "-fPIC", "-shared", "-pthread", "-I", str(d), "-I", CUDA_INCLUDE,
                    os.path.join(HERE, "sweep_harness.cpp"), "-o", str(lib_path)], check=True)
    lib = ctypes.CDLL(str(lib_path))
    F, D, I = (ctypes.POINTER(t) for t in (ctypes.c_float, ctypes.c_double, ctypes.c_int))
    lib.emu_sweep.argtypes = [I, I, ctypes.c_int, F, F, F, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, D, ctypes.c_int, F, ctypes.c_int]
    return lib


def _iv(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _internal32(a):
    return np.ascontiguousarray(a.reshape(a.shape[0], 12, -1).transpose(0, 2, 1)).astype(np.complex64)


def _oracle_layout(a):
    return np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(a.shape[0], 4, 3, -1).astype(np.complex128)


def _sap_emulated(lib, dims, block, U, kappa, eta, ncycle, nmr, mode, omegas, nclusters, oracle_mod, tinv=None,
                  Ti=None, shape=0):
    """ncycle cycles of E and O sweeps, as the library's driver launches them:
    before every sweep but the first the colour's residual eta - A psi (here
    from the oracle's operator, in place of the library's residual kernel);
    mode 3 replays the step lengths omegas[it] on every domain."""
    L = eta.shape[3]
    links = np.ascontiguousarray(U.astype(np.complex64))
    e = _internal32(eta)
    psi = np.zeros_like(e)
    ndc = int(np.prod(dims)) // int(np.prod(block)) // 2
    table = None
    if mode == 3:
        table = np.zeros((nmr, ndc, 2))
        table[..., 0] = np.real(omegas)[:, None]
        table[..., 1] = np.imag(omegas)[:, None]
    tp = table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if table is not None else None
    for cyc in range(ncycle):
        for colour in (0, 1):
            first = cyc == 0 and colour == 0
            if first:
                r = e
            else:
                p64 = _oracle_layout(psi)
                Ap = oracle_mod.apply_D(dims, U, kappa, p64) if Ti is None else oracle_mod.apply_A(dims, U, kappa,
                                                                                                    Ti, p64)
                r = _internal32(eta - Ap)
            rc = lib.emu_sweep(_iv(dims), _iv(block), colour, _fp(links), _fp(r), _fp(psi), L, kappa,
                               1 if first else 2, nmr, mode, tp, nclusters,
                               _fp(tinv) if tinv is not None else None, shape)
            assert rc == 0
    return _oracle_layout(psi)


def _rel_site(a, b):
    V = a.shape[0]
    return float(np.max(np.linalg.norm((a - b).reshape(V, -1), axis=1) / np.linalg.norm(b.reshape(V, -1), axis=1)))


CASES = [
    # dims, block, L, ncycle, nmr, clusters
    ((8, 8, 8, 8), (4, 4, 4, 4), 3, 2, 3, 5),
    ((16, 16, 16, 16), (8, 8, 8, 8), 1, 1, 2, 3),
]


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,nclusters", CASES)
@pytest.mark.parametrize("mode", [0, 3])
def test_fused_sweep_matches_oracle(sweep, oracle_mod, dims, block, L, ncycle, nmr, nclusters, mode):
    U = synth.su3_links(dims, 0.5, seed=71)
    eta = synth.gaussian_source(dims, L, seed=72)
    kappa = 0.125
    omegas = np.array([0.9 + 0.05j, 1.1 - 0.02j, 0.95 + 0.01j])[:nmr]
    got = _sap_emulated(sweep, dims, block, U, kappa, eta, ncycle, nmr, mode, omegas, nclusters, oracle_mod)
    assert not np.isnan(got).any()
    if mode == 0:
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=oracle_mod.MR_COLUMN)
    else:
        nd = int(np.prod(dims)) // int(np.prod(block))
        table = np.ascontiguousarray(np.broadcast_to(omegas[None, None, :, None], (ncycle, 2, nmr, nd)))
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=oracle_mod.MR_FROZEN,
                             omega_table=table.copy())
    assert _rel_site(got, ref) < 1e-5


@pytest.mark.parametrize("mode", [0, 3])
def test_sweep_shapes_are_bit_identical(sweep, oracle_mod, mode):
    """8^4 domains on clusters of 8 CTAs (one column per thread) and of 16
    CTAs (two columns per thread, or one): every shape sums a column's hops
    in the same order, so with frozen step lengths (mode 3, the solver's) the
    results agree bit for bit; per-column MR (mode 0) sums its dot products
    over the CTAs of a cluster, which cover other sites in each shape, so its
    step lengths and results agree to rounding.  L = 3 leaves the two-column
    shape a last group with one column."""
    dims, block, L, ncycle, nmr, nclusters = (16, 16, 16, 16), (8, 8, 8, 8), 3, 1, 2, 3
    U = synth.su3_links(dims, 0.5, seed=73)
    eta = synth.gaussian_source(dims, L, seed=74)
    omegas = np.array([0.9 + 0.05j, 1.1 - 0.02j])
    got = [_sap_emulated(sweep, dims, block, U, 0.125, eta, ncycle, nmr, mode, omegas, nclusters, oracle_mod,
                         shape=sh) for sh in (0, 1, 2)]
    if mode == 3:
        assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])
    else:
        ref = oracle_mod.sap(dims, block, U, 0.125, ncycle, nmr, eta, mr_mode=oracle_mod.MR_COLUMN)
        for g in got:
            assert _rel_site(g, ref) < 1e-5
            assert _rel_site(g, got[0]) < 1e-6


def _pack_herm(M):
    """(V, 12, 12) Hermitian, block diagonal in chirality -> the library's packed
    FP32 form: per block 6 real diagonal entries, then the entries above the
    diagonal row by row as (re, im)."""
    V = M.shape[0]
    P = np.zeros((V, 72), np.float32)
    for b in range(2):
        o = 36 * b
        for i in range(6):
            P[:, o + i] = M[:, 6 * b + i, 6 * b + i].real
        k = 6
        for i in range(6):
            for j in range(i + 1, 6):
                P[:, o + k] = M[:, 6 * b + i, 6 * b + j].real
                P[:, o + k + 1] = M[:, 6 * b + i, 6 * b + j].imag
                k += 2
    return np.ascontiguousarray(P)


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,nclusters", CASES)
@pytest.mark.parametrize("mode", [0, 3])
def test_fused_sweep_with_clover_matches_oracle(sweep, oracle_mod, dims, block, L, ncycle, nmr, nclusters, mode):
    """The Jacobi-preconditioned clover matrix A = T^{-1} D_c in the sweep."""
    U = synth.su3_links(dims, 0.5, seed=73)
    eta = synth.gaussian_source(dims, L, seed=74)
    kappa = 0.125
    Ti = oracle_mod.clover_inverse(oracle_mod.clover(dims, U, kappa, 1.3))
    omegas = np.array([0.9 + 0.05j, 1.1 - 0.02j, 0.95 + 0.01j])[:nmr]
    got = _sap_emulated(sweep, dims, block, U, kappa, eta, ncycle, nmr, mode, omegas, nclusters, oracle_mod,
                        tinv=_pack_herm(Ti), Ti=Ti)
    assert not np.isnan(got).any()
    if mode == 0:
        ref = oracle_mod.sap_ext(dims, block, U, kappa, ncycle, eta, Tinv=Ti, solver=oracle_mod.DOMAIN_MR, nmr=nmr,
                                 mr_mode=oracle_mod.MR_COLUMN)
    else:
        nd = int(np.prod(dims)) // int(np.prod(block))
        table = np.ascontiguousarray(np.broadcast_to(omegas[None, None, :, None], (ncycle, 2, nmr, nd)))
        ref = oracle_mod.sap_ext(dims, block, U, kappa, ncycle, eta, Tinv=Ti, solver=oracle_mod.DOMAIN_MR, nmr=nmr,
                                 mr_mode=oracle_mod.MR_FROZEN, omega_table=table.copy())
    assert _rel_site(got, ref) < 1e-5
