"""The CUDA path's own FP64 kernels, compiled for the host and run once per
emulated thread, against the oracle: the operator (Sec. 2.1), the SAP
pieces (Sec. 2.2: the colour residual, the Dirichlet domain operator and the
MR update) and the clover term with its Jacobi preconditioning (Sec. 2.2).  This checks the kernels' arithmetic and index maps on a machine
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

import emulation_sources
import synth
from lattice_helpers import domain_colour

HERE = os.path.join(emulation_sources.ROOT, "tests", "host_emulation")
CUDA_INCLUDE = "/usr/local/cuda/include"

# (namespace, file, start marker, end marker) of the device code to emulate
PARTS = [
    ("emu_dslash", "dslash.cu", "namespace {", emulation_sources.DSLASH_SEQ_END),
    ("emu_sap", "sap.cu", "namespace {", "}  // namespace\n"),
    ("emu_clover", "clover.cu", "namespace {", "}  // namespace\n"),
    ("emu_half", "half.cu", "namespace {", "}  // namespace\n"),
]


def _device_parts():
    # common.cuh with its inline-PTX spinor loads and stores written as plain C++
    common = emulation_sources.read("common.cuh")
    common = emulation_sources.replace_body(
        common, "__device__ __forceinline__ void load_spinor(const cx<float>* p, Spinor<float>& s)",
        "{ for (int k = 0; k < 12; ++k) (&s.c[0][0])[k] = p[k]; }")
    common = emulation_sources.replace_body(
        common, "__device__ __forceinline__ void store_spinor(cx<float>* p, const Spinor<float>& s)",
        "{ for (int k = 0; k < 12; ++k) p[k] = (&s.c[0][0])[k]; }")
    out = ['#include "shim.h"', "#include <cuda_fp16.h>", "#include <cstring>", common, "namespace mbicg {"]
    for ns, name, start, end in PARTS:
        out += [f"namespace {ns} {{", emulation_sources.cut(emulation_sources.read(name), start, end), "}"]
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
    F = ctypes.POINTER(ctypes.c_float)
    lib.emu_dslash.argtypes = [I, D, D, D, ctypes.c_int, ctypes.c_double, D, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.emu_segment_of.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.emu_clover_field.argtypes = [I, D, ctypes.c_double, D]
    lib.emu_clover_terms.argtypes = [ctypes.c_longlong, D, ctypes.c_double, D, F, F]
    lib.emu_clover_abi.argtypes = [ctypes.c_longlong, ctypes.c_int, D, D, D]
    lib.emu_nslot.argtypes = [I, I]
    lib.emu_slot.argtypes = [I, I, ctypes.c_int, ctypes.c_int, I, I]
    lib.emu_sap_residual.argtypes = [I, I, D, ctypes.c_int, D, D, D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     D]
    lib.emu_sap_domain_apply.argtypes = [I, I, D, ctypes.c_int, D, D, ctypes.c_int, ctypes.c_double, D]
    lib.emu_ssor_level.argtypes = [I, I, D, D, ctypes.c_int, D, D, ctypes.c_int, ctypes.c_double, I, ctypes.c_int,
                                   ctypes.c_int]
    lib.emu_ssor_combine.argtypes = [I, I, ctypes.c_int, D, D, D, D, D, ctypes.c_int, ctypes.c_double]
    lib.emu_colour_add.argtypes = [I, I, ctypes.c_int, D, D, ctypes.c_int]
    lib.emu_half_operator.argtypes = [I, D, D, D, ctypes.c_int, ctypes.c_double]
    lib.emu_mr_update.argtypes = [I, I, ctypes.c_int, D, D, D, D, D, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _iv(v):
    return (ctypes.c_int * 4)(*[int(x) for x in v])


def _internal(a):
    """(V, 4, 3, L) oracle layout -> the library's internal [site][rhs][12]."""
    return np.ascontiguousarray(a.reshape(a.shape[0], 12, -1).transpose(0, 2, 1))


def _oracle_layout(a):
    return np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(a.shape[0], 4, 3, -1)


@pytest.mark.parametrize("dims,L,S", [((4, 4, 4, 4), 3, 1), ((6, 2, 4, 10), 2, 4), ((2, 2, 2, 2), 5, 2),
                                      ((8, 4, 2, 6), 1, 32), ((8, 4, 4, 16), 12, 32), ((8, 2, 2, 8), 4, 8)])
def test_operator_kernel_matches_oracle(emu, oracle_mod, dims, L, S):
    """S sites per CTA as the library launches it (time-slab order where the
    segments tile the time slices: the last two cases)."""
    U = np.ascontiguousarray(synth.su3_links(dims, 0.5, seed=91))
    psi = synth.gaussian_source(dims, L, seed=92)
    kappa = 0.1375
    a = _internal(psi)
    out = np.full_like(a, np.nan)
    emu.emu_dslash(_iv(dims), _dp(U), _dp(a), _dp(out), L, kappa, None, 0, S, 1)
    ref = oracle_mod.apply_D(dims, U, kappa, psi)
    assert np.max(np.abs(_oracle_layout(out) - ref)) < 1e-14 * np.max(np.abs(ref))


def test_operator_launch_configurations_are_bit_identical(emu, oracle_mod):
    """Every configuration the autotuner may choose (sites per CTA, CTA order)
    gives the same result bit for bit."""
    dims, L = (8, 4, 4, 16), 3
    U = np.ascontiguousarray(synth.su3_links(dims, 0.5, seed=99))
    a = _internal(synth.gaussian_source(dims, L, seed=100))
    outs = []
    for S in (32, 16, 8):
        for order in (0, 1):
            out = np.full_like(a, np.nan)
            emu.emu_dslash(_iv(dims), _dp(U), _dp(a), _dp(out), L, 0.13, None, 0, S, order)
            outs.append(out)
    assert all(np.array_equal(o, outs[0]) for o in outs[1:])
    ref = oracle_mod.apply_D(dims, U, 0.13, _oracle_layout(a))
    assert np.max(np.abs(_oracle_layout(outs[0]) - ref)) < 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("wslice,tt,nt", [(32, 8, 64), (1, 8, 16), (7, 8, 24), (5, 1, 3)])
def test_segment_order_is_a_permutation_with_near_t_neighbours(emu, wslice, tt, nt):
    """Every segment is taken once; within a slab a segment's t +- 1 neighbours
    are taken within one slab's worth of CTAs of it."""
    n = wslice * nt
    seg = np.array([emu.emu_segment_of(b, wslice, tt) for b in range(n)])
    assert sorted(seg) == list(range(n))
    if tt > 1:
        pos = np.empty(n, int)
        pos[seg] = np.arange(n)
        t, w = seg // wslice, seg % wslice
        inner = (t % tt) != tt - 1                     # t + 1 in the same slab
        nxt = (t + 1) * wslice + w
        assert np.all(np.abs(pos[nxt[inner]] - pos[seg[inner]]) == 1)


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


def _sap(emu, dims, block, U, kappa, eta, ncycle, nmr, mode, tinv=None):
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
                                 int(cyc == 0 and colour == 0), _dp(tinv))
            for it in range(nmr):
                emu.emu_sap_domain_apply(_iv(dims), _iv(block), _dp(U), colour, _dp(r), _dp(q), L, kappa, _dp(tinv))
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


# ---------------------------------------------------------------------------
# clover term and Jacobi preconditioning
# ---------------------------------------------------------------------------
def _herm_off(i, j):
    return 6 + 2 * (i * 6 - i * (i + 1) // 2 + (j - i - 1))


def _unpack(P):
    """Packed per-site Hermitian chirality blocks (72 reals) -> (V, 12, 12)."""
    V = P.shape[0]
    M = np.zeros((V, 12, 12), complex)
    for b in range(2):
        blk = P[:, 36 * b:36 * b + 36].astype(np.float64)
        for i in range(6):
            M[:, 6 * b + i, 6 * b + i] = blk[:, i]
            for j in range(i + 1, 6):
                o = _herm_off(i, j)
                v = blk[:, o] + 1j * blk[:, o + 1]
                M[:, 6 * b + i, 6 * b + j] = v
                M[:, 6 * b + j, 6 * b + i] = np.conj(v)
    return M


@pytest.fixture(scope="module")
def clover_case(emu, oracle_mod):
    dims, kappa, csw = (4, 4, 2, 4), 0.13, 1.3
    V = int(np.prod(dims))
    U = np.ascontiguousarray(synth.su3_links(dims, 0.5, seed=95))
    C = np.zeros((V, 72))
    emu.emu_clover_field(_iv(dims), _dp(U), csw, _dp(C))
    Ti64 = np.zeros((V, 72))
    Ti32 = np.zeros((V, 72), np.float32)
    C32 = np.zeros((V, 72), np.float32)
    st = emu.emu_clover_terms(V, _dp(C), kappa, _dp(Ti64), Ti32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              C32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    T = oracle_mod.clover(dims, U, kappa, csw)
    return dict(dims=dims, kappa=kappa, V=V, U=U, C=C, Ti64=Ti64, Ti32=Ti32, C32=C32, status=st, T=T,
                Ti=oracle_mod.clover_inverse(T))


def test_clover_field_and_inverse_kernels(clover_case):
    c = clover_case
    assert c["status"] == 0
    assert np.max(np.abs(np.eye(12) + c["kappa"] * _unpack(c["C"]) - c["T"])) < 1e-15
    assert np.max(np.abs(_unpack(c["Ti64"]) - c["Ti"])) < 1e-14
    assert np.max(np.abs(_unpack(c["Ti32"]) - c["Ti"])) < 1e-6
    assert np.max(np.abs(c["C32"] - c["C"])) < 1e-6 * np.max(np.abs(c["C"]))


def test_clover_operator_kernels(emu, oracle_mod, clover_case):
    c = clover_case
    dims, kappa, V, U = c["dims"], c["kappa"], c["V"], c["U"]
    psi = synth.gaussian_source(dims, 3, seed=96)
    a = _internal(psi)
    out = np.zeros_like(a)
    emu.emu_dslash(_iv(dims), _dp(U), _dp(a), _dp(out), 3, kappa, _dp(c["Ti64"]), 1, 32, 0)
    ref = oracle_mod.apply_A(dims, U, kappa, c["Ti"], psi)
    assert np.max(np.abs(_oracle_layout(out) - ref)) < 1e-14 * np.max(np.abs(ref))
    emu.emu_dslash(_iv(dims), _dp(U), _dp(a), _dp(out), 3, kappa, _dp(c["C"]), 2, 32, 0)
    ref = oracle_mod.apply_clover_D(dims, U, kappa, c["T"], psi)
    assert np.max(np.abs(_oracle_layout(out) - ref)) < 1e-14 * np.max(np.abs(ref))
    # T^{-1} on an ABI-layout block (the right-hand side of the solve)
    o2 = np.zeros_like(psi)
    emu.emu_clover_abi(V, 3, _dp(c["Ti64"]), _dp(psi), _dp(o2))
    ref = np.einsum("vrc,vci->vri", c["Ti"], psi.reshape(V, 12, 3)).reshape(psi.shape)
    assert np.max(np.abs(o2 - ref)) < 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("mode", [0, 1])
def test_clover_sap_kernels(emu, oracle_mod, clover_case, mode):
    c = clover_case
    block = (2, 2, 1, 2)
    eta = synth.gaussian_source(c["dims"], 2, seed=97)
    got = _sap(emu, c["dims"], block, c["U"], c["kappa"], eta, 2, 3, mode, tinv=c["Ti64"])
    ref = oracle_mod.sap_ext(c["dims"], block, c["U"], c["kappa"], 2, eta, Tinv=c["Ti"],
                             solver=oracle_mod.DOMAIN_MR, nmr=3, mr_mode=mode)
    assert np.max(np.abs(got - ref)) < 1e-14 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# SSOR domain solves
# ---------------------------------------------------------------------------
def _levels(block):
    """Local site indices of a domain (x fastest) grouped by lx + ly + lz + lt."""
    bx, by, bz, bt = block
    n = bx * by * bz * bt
    lev = [[] for _ in range(bx + by + bz + bt - 3)]
    for l in range(n):
        x, y, z, t = l % bx, (l // bx) % by, (l // (bx * by)) % bz, l // (bx * by * bz)
        lev[x + y + z + t].append(l)
    return [np.array(v, dtype=np.int32) for v in lev]


def _ssor_colour(emu, dims, block, U, tinv, colour, y, kappa, nssor, omega):
    """B y on the domains of one colour with the emulated kernels, launched in
    the order of the library's SSOR driver."""
    L = y.shape[1]
    lev = _levels(block)
    acc, term, qv, pv, pqv, out = (np.zeros_like(y) for _ in range(6))

    def substitute(fwd, src, dst):
        for k in (range(len(lev) - 1, -1, -1) if fwd else range(len(lev))):
            loc = lev[k]
            emu.emu_ssor_level(_iv(dims), _iv(block), _dp(U), _dp(tinv), colour, _dp(src), _dp(dst), L,
                               kappa * omega, loc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(loc), int(fwd))

    substitute(True, y, acc)
    term[...] = acc
    for _ in range(nssor):
        substitute(False, term, qv)
        substitute(True, term, pv)
        substitute(True, qv, pqv)
        emu.emu_ssor_combine(_iv(dims), _iv(block), colour, _dp(pv), _dp(qv), _dp(pqv), _dp(term), _dp(acc), L,
                             omega)
    substitute(False, acc, out)
    return out


@pytest.mark.parametrize("clover", [False, True])
@pytest.mark.parametrize("nssor,omega", [(0, 1.0), (1, 1.26), (2, 0.9)])
def test_ssor_domain_kernels(emu, oracle_mod, clover_case, clover, nssor, omega):
    c = clover_case
    dims, block = c["dims"], (2, 2, 1, 2)
    tinv = c["Ti64"] if clover else None
    y = synth.gaussian_source(dims, 2, seed=98)
    col = domain_colour(dims, block)
    for colour in (0, 1):
        got = _oracle_layout(_ssor_colour(emu, dims, block, c["U"], tinv, colour, _internal(y), c["kappa"],
                                          nssor, omega))
        ref = oracle_mod.ssor_domains(dims, block, c["U"], c["kappa"], nssor, omega, colour, y,
                                      Tinv=c["Ti"] if clover else None)
        on = col == colour
        assert np.max(np.abs(got[on] - ref[on])) < 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("clover", [False, True])
def test_ssor_sap_kernels(emu, oracle_mod, clover_case, clover):
    """M_SAP with SSOR domain solves: per colour the residual kernel, the SSOR
    solve and psi += x, in the order of the library's driver."""
    c = clover_case
    dims, block, kappa = c["dims"], (2, 2, 1, 2), c["kappa"]
    tinv = c["Ti64"] if clover else None
    eta = synth.gaussian_source(dims, 2, seed=99)
    e = _internal(eta)
    psi, r = np.zeros_like(e), np.zeros_like(e)
    L = e.shape[1]
    for cyc in range(2):
        for colour in (0, 1):
            emu.emu_sap_residual(_iv(dims), _iv(block), _dp(c["U"]), colour, _dp(e), _dp(psi), _dp(r), L, kappa,
                                 int(cyc == 0 and colour == 0), _dp(tinv))
            x = _ssor_colour(emu, dims, block, c["U"], tinv, colour, r, kappa, 1, 1.26)
            emu.emu_colour_add(_iv(dims), _iv(block), colour, _dp(x), _dp(psi), L)
    ref = oracle_mod.sap_ext(dims, block, c["U"], kappa, 2, eta, Tinv=c["Ti"] if clover else None,
                             solver=oracle_mod.DOMAIN_SSOR, nssor=1, omega=1.26)
    assert np.max(np.abs(_oracle_layout(psi) - ref)) < 1e-14 * np.max(np.abs(ref))
# FP16 storage (half.cu)
# ---------------------------------------------------------------------------
def _comps(a):
    """(V, 4, 3, L) complex -> (V, L, 24) reals of each (site, rhs) spinor."""
    V, L = a.shape[0], a.shape[-1]
    return np.stack([a.real, a.imag], -1).reshape(V, 12, L, 2).transpose(0, 2, 1, 3).reshape(V, L, 24)


def _half_operator(emu, dims, U, psi, kappa):
    out = np.zeros_like(psi)
    emu.emu_half_operator(_iv(dims), _dp(np.ascontiguousarray(U)), _dp(np.ascontiguousarray(psi)), _dp(out),
                          psi.shape[3], kappa)
    return out


@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 3), ((6, 2, 4, 10), 2)])
def test_fp16_kernels_round_trip_is_the_oracle_format(emu, oracle_mod, dims, L):
    """kappa = 0: ABI -> FP16 storage -> operator -> ABI is the input as the
    oracle's FP16 format represents it, bit for bit (a zero spinor included)."""
    U = synth.su3_links(dims, 0.5, seed=95)
    psi = synth.gaussian_source(dims, L, seed=96)
    psi[3] = 0
    assert np.array_equal(_half_operator(emu, dims, U, psi, 0.0), oracle_mod.quantize_fp16(psi))


@pytest.mark.parametrize("dims,L", [((4, 4, 4, 4), 3), ((6, 2, 4, 10), 2)])
def test_fp16_operator_kernel_matches_oracle(emu, oracle_mod, dims, L):
    """The oracle on the FP16-represented links and input, rounded into the
    FP16 format: equal up to one FP16 step of the output scale."""
    U = synth.su3_links(dims, 0.5, seed=97)
    psi = synth.gaussian_source(dims, L, seed=98)
    kappa = 0.13
    got = _half_operator(emu, dims, U, psi, kappa)
    exp = oracle_mod.quantize_fp16(oracle_mod.apply_D(dims, oracle_mod.quantize_links_fp16(U), kappa,
                                                      oracle_mod.quantize_fp16(psi)))
    g, e = _comps(got), _comps(exp)
    s = np.abs(e).max(axis=2, keepdims=True)
    assert np.all(np.abs(g - e) <= 2.0 ** -10 * s)
    assert np.mean(np.abs(g - e) > 2.0 ** -20 * s) < 0.05
