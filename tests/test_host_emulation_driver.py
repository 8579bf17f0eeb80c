"""The library's SAP driver (Sec. 2.2) end to end on the CPU: sap_apply and
the launchers and kernels it uses, the host code being the library's own
(its launches rewritten onto the threaded emulator by
tests/emulation_sources.py), against the oracle's SAP: the FP64 multi-kernel
path with per-column and block-shared MR, the FP32 fused cluster sweep and
the FP32 multi-kernel path, and the frozen step lengths: recorded by the
driver (their table compared entry by entry with the oracle's), then replayed
by the fused sweep."""
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
DIMS, BLOCK, L, KAPPA, NCYCLE, NMR = (8, 8, 8, 8), (4, 4, 4, 4), 2, 0.125, 2, 3


@pytest.fixture(scope="module")
def drv(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INCLUDE, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("driver_emulation")
    (d / "driver_parts.inc").write_text(emulation_sources.driver_parts())
    for f in ("shim_threads.h", "emu_runtime.h"):
        shutil.copy(os.path.join(HERE, f), d / f)
    lib_path = d / "libdrv.so"
    subprocess.run(["g++", "-std=c++20", "-O1", "-fPIC", "-shared", "-pthread", "-I", str(d), "-I", CUDA_INCLUDE,
                    os.path.join(HERE, "sap_driver_harness.cpp"), "-o", str(lib_path)], check=True)
    lib = ctypes.CDLL(str(lib_path))
    V, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.emu_sap_apply.argtypes = [ctypes.c_int, I, I, V, V, V, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, D, I]
    lib.emu_colour_domain.argtypes = [I, I, ctypes.c_int, ctypes.c_int]
    return lib


@pytest.fixture(scope="module")
def problem():
    return synth.su3_links(DIMS, 0.5, seed=71), synth.gaussian_source(DIMS, L, seed=72)


def _iv(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _internal(a, dt):
    return np.ascontiguousarray(a.reshape(a.shape[0], 12, -1).transpose(0, 2, 1)).astype(dt)


def _oracle_layout(a):
    return np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(a.shape[0], 4, 3, -1).astype(np.complex128)


def _sap(drv, U, eta, fp64, mode, fused, monkeypatch, table=None):
    monkeypatch.setenv("MBICG_SAP_FUSED", "1" if fused else "0")
    dt = np.complex128 if fp64 else np.complex64
    links = np.ascontiguousarray(U.astype(dt))
    e = _internal(eta, dt)
    psi = np.zeros_like(e)
    unset = ctypes.c_int(0)
    tp = table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if table is not None else None
    n = drv.emu_sap_apply(fp64, _iv(DIMS), _iv(BLOCK), ctypes.c_void_p(links.ctypes.data),
                          ctypes.c_void_p(e.ctypes.data), ctypes.c_void_p(psi.ctypes.data), L, KAPPA, NCYCLE, NMR,
                          mode, tp, ctypes.byref(unset))
    assert n > 0
    return _oracle_layout(psi), n, unset.value


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("fp64,fused,mode,tol", [(1, True, 0, 1e-13), (1, True, 1, 1e-13), (0, True, 0, 1e-6),
                                                 (0, False, 0, 1e-6), (0, False, 1, 1e-6)])
def test_driver_matches_oracle(drv, oracle_mod, problem, monkeypatch, fp64, fused, mode, tol):
    U, eta = problem
    got, launches, _ = _sap(drv, U, eta, fp64, mode, fused, monkeypatch)
    ref = oracle_mod.sap(DIMS, BLOCK, U, KAPPA, NCYCLE, NMR, eta, mr_mode=mode)
    assert _rel(got, ref) < tol
    # the fused sweep is one launch per colour sweep (FP32, modes 0 and 3), the
    # residual kernel one before every sweep but the first
    assert (launches == 2 * NCYCLE + 2 * NCYCLE - 1) == (fp64 == 0 and fused and mode == 0)


def test_frozen_step_lengths_record_and_replay(drv, oracle_mod, problem, monkeypatch):
    U, eta = problem
    nd = int(np.prod(DIMS)) // int(np.prod(BLOCK))
    ndc = nd // 2
    table = np.full((NCYCLE, 2, NMR, ndc, 2), np.nan)
    got, _, unset = _sap(drv, U, eta, 1, 2, True, monkeypatch, table)   # recording: multi-kernel, FP64
    otab = np.full((NCYCLE, 2, NMR, nd), np.nan + 0j)
    ref = oracle_mod.sap(DIMS, BLOCK, U, KAPPA, NCYCLE, NMR, eta, mr_mode=oracle_mod.MR_FROZEN, omega_table=otab)
    assert unset == 0 and not np.isnan(table).any()
    assert _rel(got, ref) < 1e-13
    for colour in (0, 1):
        for k in range(ndc):
            lex = drv.emu_colour_domain(_iv(DIMS), _iv(BLOCK), colour, k)
            rec = table[:, colour, :, k, 0] + 1j * table[:, colour, :, k, 1]
            assert np.max(np.abs(rec - otab[:, colour, :, lex])) < 1e-12 * np.nanmax(np.abs(otab))
    # replay in FP32 by the fused sweep (mode 3) with the recorded table
    got32, launches, _ = _sap(drv, U, eta, 0, 3, True, monkeypatch, table.copy())
    assert launches == 2 * NCYCLE + 2 * NCYCLE - 1
    assert _rel(got32, ref) < 1e-6
