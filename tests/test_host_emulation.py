"""The CUDA path's own FP64 kernels, compiled for the host and run once per
emulated thread, against the oracle: the operator (Sec. 2.1) and the SAP
pieces (Sec. 2.2: the colour residual, the Dirichlet domain operator and the
MR update).  This checks the kernels' arithmetic and index maps on a machine
without a GPU; the launch configurations, the FP32 and fused kernels and the
device memory handling are covered by the -m gpu tests.

The kernels and their device helpers are cut out of the CUDA sources between
fixed markers (no launches) and compiled with g++ against tests/host_emulation/
shim.h; the oracle shares nothing with them."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from lattice_helpers import domain_colour

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1104_0737_gb300", "csrc")
HERE = os.path.join(ROOT, "tests", "host_emulation")
CUDA_INCLUDE = "/usr/local/cuda/include"

# (file, start marker, end marker) of the device code each namespace gets
PARTS = [
    ("emu_dslash", "dslash.cu", "namespace {",
     "// ---------------------------------------------------------------------------\n// Fused SAP colour sweep"),
    ("emu_sap", "sap.cu", "namespace {", "}  // namespace\n\ntemplate <typename R>\nvoid sap_apply("),
]


def _device_parts():
    out = ['#include "shim.h"', f'#include "{os.path.join(CSRC, "common.cuh")}"', "namespace mbicg {"]
    for ns, name, start, end in PARTS:
        with open(os.path.join(CSRC, name)) as f:
            s = f.read()
        a = s.index(start)
        b = s.index(end, a)
        out += [f"namespace {ns} {{", s[a + len(start):b], "}"]
    out.append("}")
    return "\n".join(out)


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INCLUDE, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("host_emulation")
    (d / "device_parts.inc").write_text(_device_parts())
    shutil.copy(os.path.join(HERE, "shim.h"), d / "shim.h")
    lib_path = d / "libemu.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I", str(d), "-I", CUDA_INCLUDE,
                    os.path.join(HERE, "harness.cpp"), "-o", str(lib_path)], check=True)
    lib = ctypes.CDLL(str(lib_path))
    D, I = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.emu_dslash.argtypes = [I, D, D, D, ctypes.c_int, ctypes.c_double]
    lib.emu_nslot.argtypes = [I, I]
    lib.emu_slot.argtypes = [I, I, ctypes.c_int, ctypes.c_int, I, I]
    lib.emu_sap_residual.argtypes = [I, I, D, ctypes.c_int, D, D, D, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.emu_sap_domain_apply.argtypes = [I, I, D, ctypes.c_int, D, D, ctypes.c_int, ctypes.c_double]
    lib.emu_mr_update.argtypes = [I, I, ctypes.c_int, D, D, D, D, D, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iv(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _internal(a):
    """(V, 4, 3, L) oracle layout -> the library's internal [site][rhs][12]."""
    return np.ascontiguousarray(a.reshape(a.shape[0], 12, -1).transpose(0, 2, 1))


def _oracle_layout(a):
    return np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(a.shape[0], 4, 3, -1)


@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 3), ((6, 2, 4, 10), 2), ((2, 2, 2, 2), 5), ((8, 4, 2, 6), 1)])
def test_operator_kernel_matches_oracle(emu, oracle_mod, dims, L):
    U = np.ascontiguousarray(synth.su3_links(dims, 0.5, seed=91))
    psi = synth.gaussian_source(dims, L, seed=92)
    kappa = 0.1375
    a = _internal(psi)
    out = np.zeros_like(a)
    emu.emu_dslash(_iv(dims), _dp(U), _dp(a), _dp(out), L, kappa)
    ref = oracle_mod.apply_D(dims, U, kappa, psi)
    assert np.max(np.abs(_oracle_layout(out) - ref)) < 1e-14 * np.max(np.abs(ref))


def _slots(emu, dims, block, colour):
    n = emu.emu_nslot(_iv(dims), _iv(block))
    out = []
    for sl in range(n):
        s, k = ctypes.c_int(), ctypes.c_int()
        emu.emu_slot(_iv(dims), _iv(block), colour, sl, ctypes.byref(s), ctypes.byref(k))
        out.append((s.value, k.value))
    return out


@pytest.mark.parametrize("dims,block", [((4, 4, 2, 4), (2, 2, 1, 2)), ((8, 4, 4, 4), (4, 2, 2, 2))])
def test_slot_map_covers_each_colour_once(emu, dims, block):
    """The slots of a colour visit every site of that colour's domains exactly
    once, and a domain's slots are contiguous."""
    col = domain_colour(dims, block)
    Vd = int(np.prod(block))
    for colour in (0, 1):
        sl = _slots(emu, dims, block, colour)
        sites = np.array([s for s, _ in sl])
        assert sorted(sites) == sorted(np.nonzero(col == colour)[0])
        ks = np.array([k for _, k in sl])
        assert np.array_equal(ks, np.repeat(np.arange(len(sl) // Vd), Vd))


def _sap(emu, dims, block, U, kappa, eta, ncycle, nmr, mode):
    """psi = M_SAP eta with the emulated kernels, launched in the order of the
    library's multi-kernel SAP driver; the step lengths are formed here from
    the emulated q and r (per column, or shared by the columns)."""
    V, L = eta.shape[0], eta.shape[3]
    e = _internal(eta)
    psi, r, q, x = (np.zeros_like(e) for _ in range(4))
    ndc = V // int(np.prod(block)) // 2
    for cyc in range(ncycle):
        for colour in (0, 1):
            sl = _slots(emu, dims, block, colour)
            emu.emu_sap_residual(_iv(dims), _iv(block), _dp(U), colour, _dp(e), _dp(psi), _dp(r), L, kappa,
                                 int(cyc == 0 and colour == 0))
            for it in range(nmr):
                emu.emu_sap_domain_apply(_iv(dims), _iv(block), _dp(U), colour, _dp(r), _dp(q), L, kappa)
                num = np.zeros((ndc, L), complex)
                den = np.zeros((ndc, L))
                for s, k in sl:
                    num[k] += np.sum(np.conj(q[s]) * r[s], axis=1)
                    den[k] += np.sum(np.abs(q[s]) ** 2, axis=1)
                if mode == 1:
                    num = np.repeat(num.sum(1, keepdims=True), L, 1)
                    den = np.repeat(den.sum(1, keepdims=True), L, 1)
                om = np.where(den > 0, num / np.where(den > 0, den, 1), 0)
                omega = np.ascontiguousarray(np.stack([om.real, om.imag], -1))
                emu.emu_mr_update(_iv(dims), _iv(block), colour, _dp(omega), _dp(r), _dp(q), _dp(x), _dp(psi), L,
                                  int(it == 0), int(it == nmr - 1))
    return _oracle_layout(psi)


@pytest.mark.parametrize("mode", [0, 1])
def test_sap_kernels_match_oracle(emu, oracle_mod, mode):
    dims, block = (4, 4, 2, 4), (2, 2, 1, 2)
    U = np.ascontiguousarray(synth.su3_links(dims, 0.5, seed=93))
    eta = synth.gaussian_source(dims, 2, seed=94)
    got = _sap(emu, dims, block, U, 0.13, eta, 2, 3, mode)
    ref = oracle_mod.sap(dims, block, U, 0.13, 2, 3, eta, mr_mode=mode)
    assert np.max(np.abs(got - ref)) < 1e-14 * np.max(np.abs(ref))
