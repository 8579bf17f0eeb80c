"""The autotuner's host code (paper_1104_0737_gb300/csrc/tune.cu, compiled
with g++): the table picks the smallest median time, skips unusable
candidates, measures a key once, survives a save/load round trip and
concurrent use; the operator's candidate configurations respect the thread
limit and use the time-slab order only where it applies.  That the
candidates give bit-identical results is checked through the operator's host
emulation (test_host_emulation.py)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import emulation_sources

HERE = os.path.join(emulation_sources.ROOT, "tests", "host_emulation")


@pytest.fixture(scope="module")
def tune(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is missing")
    d = tmp_path_factory.mktemp("tune")
    lib_path = d / "libtune.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-x", "c++",
                    os.path.join(emulation_sources.CSRC, "tune.cu"), "-x", "c++",
                    os.path.join(HERE, "tune_harness.cpp"), "-I", emulation_sources.CSRC, "-o", str(lib_path)],
                   check=True)
    lib = ctypes.CDLL(str(lib_path))
    D, I = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.tune_pick.argtypes = [ctypes.c_char_p, ctypes.c_int, D, ctypes.c_int]
    lib.tune_save.argtypes = lib.tune_load.argtypes = [ctypes.c_char_p]
    lib.tune_lookup.argtypes = [ctypes.c_char_p]
    lib.tune_candidates.argtypes = [I, ctypes.c_int, ctypes.c_int, I]
    lib.tune_key.argtypes = [ctypes.c_int, I, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.tune_sweep_key.argtypes = [ctypes.c_int, ctypes.c_int, I, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    return lib


def _pick(lib, key, times):
    t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
    return lib.tune_pick(key.encode(), t.shape[0], t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t.shape[1])


def test_pick_smallest_median_once(tune):
    # medians 2.0, 1.5 (one slow outlier), 1.6, unusable
    times = [[2.0, 2.1, 1.9], [1.5, 9.0, 1.4], [1.6, 1.6, 1.6], [-1.0, 0.1, 0.1]]
    calls0 = tune.tune_calls()
    assert _pick(tune, "k/a", times) == 1
    assert tune.tune_calls() - calls0 == 3 + 3 + 3 + 1  # the unusable candidate stops at its first run
    assert _pick(tune, "k/a", [[0.0] * 3] * 4) == 1      # known key: not measured again
    assert tune.tune_calls() - calls0 == 10
    assert _pick(tune, "k/b", [[1.0], [1.0]]) == 0       # ties: the lower index
    assert _pick(tune, "k/c", [[-1.0], [-2.0]]) == -1    # nothing usable: nothing recorded
    assert tune.tune_lookup(b"k/c") == -2


def test_save_and_load(tune, tmp_path):
    _pick(tune, "k/save", [[3.0], [1.0], [2.0]])
    path = str(tmp_path / "tune.txt").encode()
    assert tune.tune_save(path) == 1
    n = tune.tune_size()
    assert tune.tune_load(path) == n
    assert tune.tune_lookup(b"k/save") == 1
    assert tune.tune_load(b"/nonexistent/dir/file") == -1


def test_concurrent_picks(tune):
    before = tune.tune_size()
    assert tune.tune_concurrent(8, 50) == before + 50
    for k in range(50):
        assert tune.tune_lookup(f"c/{k}".encode()) == (3 - k % 3) % 3  # time (i + k) % 3 is 0 at i = -k mod 3


@pytest.mark.parametrize("dims,L,maxt", [((32, 32, 32, 64), 12, 384), ((32, 32, 32, 64), 12, 256),
                                         ((6, 2, 4, 10), 5, 384), ((8, 8, 8, 16), 16, 384), ((4, 4, 4, 4), 1, 384)])
def test_operator_candidates(tune, dims, L, maxt):
    out = (ctypes.c_int * 16)()
    n = tune.tune_candidates((ctypes.c_int * 4)(*dims), L, maxt, out)
    cand = [(out[2 * i], out[2 * i + 1]) for i in range(n)]
    sizes = sorted({S for S, _ in cand}, reverse=True)
    assert 1 <= len(sizes) <= 3
    assert all(S & (S - 1) == 0 and S * L <= maxt for S in sizes)
    assert sizes[0] * 2 * L > maxt                         # the largest size that fits comes first
    slice_ = dims[0] * dims[1] * dims[2]
    for S in sizes:
        slab_ok = slice_ % S == 0 and dims[3] % 8 == 0
        assert ((S, 1) in cand) == slab_ok and (S, 0) in cand
    buf = ctypes.create_string_buffer(128)
    tune.tune_key(4, (ctypes.c_int * 4)(*dims), L, buf, 128)
    assert buf.value.decode() == f"dslash/fp32/{dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}/L{L}"


def test_sweep_keys(tune):
    """One key per storage, operator, lattice and L for the SAP sweep's launch
    shape (8-CTA clusters; 16-CTA clusters with two columns per thread; with
    one): the keys bench.py prints under "autotuned" and MBICG_TUNE_FILE holds."""
    assert tune.tune_sweep_shapes() == 3
    buf = ctypes.create_string_buffer(128)
    dims = (ctypes.c_int * 4)(32, 32, 32, 64)
    keys = set()
    for half in (0, 1):
        for clover in (0, 1):
            for L in (1, 12):
                n = tune.tune_sweep_key(half, clover, dims, L, buf, 128)
                k = buf.value.decode()
                assert n == len(k) and k.startswith("sap_sweep/") and k.endswith(f"/32x32x32x64/L{L}")
                assert (("fp16" in k) == bool(half)) and (("clover" in k) == bool(clover))
                keys.add(k)
    assert len(keys) == 8
    tune.tune_sweep_key(0, 0, dims, 12, buf, 128)
    assert buf.value.decode() == "sap_sweep/fp32/32x32x32x64/L12"
