"""The operator's autotuner through the C ABI on the CPU: the emulated library
(tests/emulated_library.py; the emulated events read the host clock, so the
tuner really times its candidates) solves the same system without and with
MBICG_AUTOTUNE.  The tuner runs when the solver allocates its buffers: it
records one choice per precision in the file named by MBICG_TUNE_FILE, each
an index into the candidate list, and since every candidate computes the
same result the solution, the iteration count and the operator's output are
bit for bit those of the untuned run."""
import ctypes
import re

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb  # the ctypes structures only; no library is loaded
import synth

# slices of 64 sites and 8 time slices: the time-slab order applies for S = 64 and 32
DIMS, L, KAPPA = (4, 4, 4, 8), 2, 0.12
NCAND = {32: 5, 64: 5}  # FP32 (at most 384 threads) and FP64 (256): S = 128, 64+slabs, 32+slabs


def _v(a):
    return ctypes.c_void_p(a.ctypes.data)


def _run(lib, U, B, psi):
    c = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(c), (ctypes.c_int * 4)(*DIMS), 0, None) == mb.MBICG_OK
    try:
        assert lib.mbicg_load_gauge(c, _v(U)) == mb.MBICG_OK
        p = mb.mbicg_params()
        lib.mbicg_default_params(ctypes.byref(p))
        p.block = (ctypes.c_int * 4)(2, 2, 2, 4)
        X = np.empty_like(B)
        it = ctypes.c_int(0)
        tres = np.zeros(L)
        rc = lib.mbicg_block_solve(c, _v(B), _v(X), L, KAPPA, 1e-9, ctypes.byref(p), ctypes.byref(it),
                                   tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert rc == mb.MBICG_OK, lib.mbicg_last_error(c)
        y = np.empty_like(psi)
        assert lib.mbicg_apply_D(c, _v(psi), _v(y), L, KAPPA, mb.MBICG_FP32) == mb.MBICG_OK
        return X, it.value, y
    finally:
        lib.mbicg_destroy(c)


def test_tuned_solve_is_bit_identical(emulated_library, tmp_path, monkeypatch):
    lib = emulated_library
    U = synth.su3_links(DIMS, 0.5, seed=1200)
    B = synth.gaussian_source(DIMS, L, seed=1201)
    psi = synth.gaussian_source(DIMS, L, seed=1202)
    monkeypatch.delenv("MBICG_AUTOTUNE", raising=False)
    X0, it0, y0 = _run(lib, U, B, psi)

    tune_file = tmp_path / "tune.txt"
    monkeypatch.setenv("MBICG_AUTOTUNE", "1")
    monkeypatch.setenv("MBICG_TUNE_FILE", str(tune_file))
    X1, it1, y1 = _run(lib, U, B, psi)
    assert it1 == it0
    assert np.array_equal(X1, X0) and np.array_equal(y1, y0)

    lines = tune_file.read_text().split("\n")
    entries = {}
    for ln in filter(None, lines):
        key, idx = ln.rsplit(" ", 1)
        entries[key] = int(idx)
    dims = "x".join(map(str, DIMS))
    for bits, n in NCAND.items():
        key = f"dslash/fp{bits}/{dims}/L{L}"
        assert key in entries, entries
        assert 0 <= entries[key] < n
    assert all(re.fullmatch(r"dslash/fp(32|64)/\d+x\d+x\d+x\d+/L\d+", k) for k in entries)


def test_no_tuning_when_switched_off(emulated_library, tmp_path, monkeypatch):
    """MBICG_AUTOTUNE=0 tunes nothing: no file is written."""
    lib = emulated_library
    tune_file = tmp_path / "off.txt"
    monkeypatch.setenv("MBICG_AUTOTUNE", "0")
    monkeypatch.setenv("MBICG_TUNE_FILE", str(tune_file))
    dims = (4, 4, 4, 4)
    c = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(c), (ctypes.c_int * 4)(*dims), 0, None) == mb.MBICG_OK
    try:
        assert lib.mbicg_load_gauge(c, _v(synth.su3_links(dims, 0.5, seed=1203))) == mb.MBICG_OK
        p = mb.mbicg_params()
        lib.mbicg_default_params(ctypes.byref(p))
        p.block = (ctypes.c_int * 4)(2, 2, 2, 2)
        B = synth.gaussian_source(dims, 1, seed=1204)
        X = np.empty_like(B)
        it = ctypes.c_int(0)
        tres = np.zeros(1)
        assert lib.mbicg_block_solve(c, _v(B), _v(X), 1, KAPPA, 1e-8, ctypes.byref(p), ctypes.byref(it),
                                     tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == mb.MBICG_OK
    finally:
        lib.mbicg_destroy(c)
    assert not tune_file.exists()
