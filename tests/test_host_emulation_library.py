"""The whole library, host code and kernels, run on the CPU through its C ABI
(test infrastructure: built by tests/emulated_library.py into a temporary
directory from the CUDA sources, never by the package's build and never
loaded by the package).
Each CUDA source becomes a g++ translation unit (tests/emulation_sources.py:
launches rewritten onto the threaded emulator, inline PTX replaced); the few
CUDA runtime calls are emulated over host memory
(tests/host_emulation/emu_cudart.cpp; stream capture is refused, so the
solver runs its iterations eagerly).  Checked against the oracle: the
operator with host pointers in FP64 and FP32, and mbicg_block_solve in FP64
and in mixed precision (reliable updates), with dummy right-hand sides and an
initial guess, mbicg_sap_precond (per-column and block MR, FP64 and FP32),
the residual history and the per-class launch profile, the FP16-storage
operator against the oracle's FP16 format,
the allocation-free operator on emulated device buffers, the give-up path of
the bounded mbarrier wait, plus the ABI's argument errors.  This exercises the solver's
host logic of Algorithm 2 on a machine without a GPU; the -m gpu tests run the
same code on the hardware."""
import ctypes
import os

import numpy as np
import pytest

import emulation_sources
import oracle

import paper_1104_0737_gb300 as mb  # the ctypes structures only; no library is loaded
import synth

DIMS, L, KAPPA = (4, 4, 4, 4), 2, 0.12


@pytest.fixture(scope="module")
def lib(emulated_library):
    return emulated_library


@pytest.fixture(scope="module")
def ctx(lib):
    c = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(c), (ctypes.c_int * 4)(*DIMS), 0, None) == mb.MBICG_OK
    U = synth.su3_links(DIMS, 0.4, seed=1000)
    assert lib.mbicg_load_gauge(c, ctypes.c_void_p(U.ctypes.data)) == mb.MBICG_OK
    yield c, U
    lib.mbicg_destroy(c)


def _v(a):
    return ctypes.c_void_p(a.ctypes.data)


def _params(lib, **kw):
    p = mb.mbicg_params()
    lib.mbicg_default_params(ctypes.byref(p))
    p.block = (ctypes.c_int * 4)(2, 2, 2, 2)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _solve(lib, c, B, X, p, tol=1e-10):
    it = ctypes.c_int(0)
    tres = np.zeros(B.shape[3])
    rc = lib.mbicg_block_solve(c, _v(B), _v(X), B.shape[3], KAPPA, tol, ctypes.byref(p), ctypes.byref(it),
                               tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    st = mb.mbicg_stats()
    lib.mbicg_get_stats(c, ctypes.byref(st))
    return rc, it.value, tres, st


def _residual(oracle_mod, U, B, X):
    R = B - oracle_mod.apply_D(DIMS, U, KAPPA, X)
    n = B.shape[3]
    return np.linalg.norm(R.reshape(-1, n), axis=0) / np.linalg.norm(B.reshape(-1, n), axis=0)


@pytest.mark.parametrize("prec,tol", [(mb.MBICG_FP64, 1e-14), (mb.MBICG_FP32, 1e-6)])
def test_operator_through_the_abi(lib, ctx, oracle_mod, prec, tol):
    c, U = ctx
    B = synth.gaussian_source(DIMS, L, seed=2001)
    out = np.empty_like(B)
    assert lib.mbicg_apply_D(c, _v(B), _v(out), L, KAPPA, prec) == mb.MBICG_OK
    ref = oracle_mod.apply_D(DIMS, U, KAPPA, B)
    assert np.max(np.abs(out - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec_D", [mb.MBICG_FP64, mb.MBICG_FP32])
def test_block_solve_through_the_abi(lib, ctx, oracle_mod, prec_D):
    c, U = ctx
    B = synth.gaussian_source(DIMS, L, seed=2000)
    X = np.empty_like(B)
    rc, iters, tres, st = _solve(lib, c, B, X, _params(lib, prec_D=prec_D))
    assert rc == mb.MBICG_OK and iters > 0, lib.mbicg_last_error(c)
    assert np.max(tres) <= 1e-10 and np.max(_residual(oracle_mod, U, B, X)) <= 1e-10
    # the mixed-precision loop refreshes its residual with the FP64 operator
    assert (st.reliable_updates > 0) == (prec_D == mb.MBICG_FP32)
    ref = oracle_mod.block_bicgstab(DIMS, U, KAPPA, B, 1e-12, ncycle=4, nmr=4, block=(2, 2, 2, 2),
                                    mr_mode=oracle_mod.MR_FROZEN)
    assert np.max(np.abs(X - ref["X"])) < 1e-8 * np.max(np.abs(ref["X"]))


def test_dummy_columns_and_initial_guess(lib, ctx, oracle_mod):
    c, U = ctx
    B = synth.gaussian_source(DIMS, 2, seed=2002)
    X = np.empty_like(B)
    rc, _, tres, _ = _solve(lib, c, B, X, _params(lib, dummy_rhs=2, dummy_seed=7))
    assert rc == mb.MBICG_OK and np.max(_residual(oracle_mod, U, B, X)) <= 1e-10
    # restarting from the solution converges at once
    X2 = X.copy()
    rc, iters, _, _ = _solve(lib, c, B, X2, _params(lib, use_x0=1))
    assert rc == mb.MBICG_OK and iters <= 1


def test_abi_errors(lib, ctx):
    c, _ = ctx
    B = synth.gaussian_source(DIMS, 1, seed=2003)
    X = np.empty_like(B)
    assert _solve(lib, c, B, X, _params(lib), tol=0.0)[0] == mb.MBICG_EINVAL
    assert _solve(lib, c, B, X, _params(lib, block=(ctypes.c_int * 4)(4, 4, 4, 4)))[0] == mb.MBICG_EINVAL
    B0 = np.zeros_like(B)
    assert _solve(lib, c, B0, X, _params(lib))[0] == mb.MBICG_EINVAL
    Bn = B.copy()
    Bn[0, 0, 0, 0] = np.nan
    assert _solve(lib, c, Bn, X, _params(lib))[0] == mb.MBICG_ENAN
    fresh = ctypes.c_void_p()
    assert lib.mbicg_create(ctypes.byref(fresh), (ctypes.c_int * 4)(*DIMS), 0, None) == mb.MBICG_OK
    assert _solve(lib, fresh, B, X, _params(lib))[0] == mb.MBICG_ENOGAUGE
    # a field that fails to load replaces the one before it by none
    U = synth.su3_links(DIMS, 0.4, seed=1000)
    assert lib.mbicg_load_gauge(fresh, _v(U)) == mb.MBICG_OK
    Un = U.copy()
    Un[7, 2, 1, 1] = np.inf
    assert lib.mbicg_load_gauge(fresh, _v(Un)) == mb.MBICG_ENAN
    assert _solve(lib, fresh, B, X, _params(lib))[0] == mb.MBICG_ENOGAUGE
    assert lib.mbicg_load_gauge(fresh, _v(U)) == mb.MBICG_OK
    assert _solve(lib, fresh, B, X, _params(lib))[0] == mb.MBICG_OK
    lib.mbicg_destroy(fresh)


def _device_copy(lib, a):
    """An emulated device buffer (the runtime's own allocation) holding a copy of a."""
    p = ctypes.c_void_p()
    assert lib.cudaMalloc(ctypes.byref(p), a.nbytes) == 0
    ctypes.memmove(p, a.ctypes.data, a.nbytes)
    return p


def _pinned_copy(lib, a):
    """An emulated page-locked host buffer (the runtime's cudaMallocHost) holding
    a copy of a, and a numpy view of it."""
    p = ctypes.c_void_p()
    assert lib.cudaMallocHost(ctypes.byref(p), a.nbytes) == 0
    view = np.ctypeslib.as_array((ctypes.c_char * a.nbytes).from_address(p.value))
    arr = np.frombuffer(view, dtype=a.dtype).reshape(a.shape)
    arr[...] = a
    return p, arr


def test_pinned_host_blocks_take_the_mapped_copy(lib, ctx):
    """Blocks in page-locked host memory are staged by the mapped-host copy
    kernel (pageable ones by the runtime copy): the operator and a block solve
    give the same bits either way."""
    c, U = ctx
    for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
        psi = synth.gaussian_source(DIMS, 3, seed=2010)
        ref = np.empty_like(psi)
        assert lib.mbicg_apply_D(c, _v(psi), _v(ref), 3, KAPPA, prec) == mb.MBICG_OK
        pin, pin_arr = _pinned_copy(lib, psi)
        pout, pout_arr = _pinned_copy(lib, np.zeros_like(psi))
        assert lib.mbicg_apply_D(c, pin, pout, 3, KAPPA, prec) == mb.MBICG_OK
        assert np.array_equal(pout_arr, ref)
        lib.cudaFreeHost(pin)
        lib.cudaFreeHost(pout)
    B = synth.gaussian_source(DIMS, L, seed=2011)
    X = np.empty_like(B)
    assert _solve(lib, c, B, X, _params(lib))[0] == mb.MBICG_OK
    pB, B_arr = _pinned_copy(lib, B)
    pX, X_arr = _pinned_copy(lib, np.zeros_like(B))
    it = ctypes.c_int(0)
    tres = np.zeros(L)
    p = _params(lib)
    assert lib.mbicg_block_solve(c, pB, pX, L, KAPPA, 1e-10, ctypes.byref(p), ctypes.byref(it),
                                 tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == mb.MBICG_OK
    assert np.array_equal(X_arr, X)
    lib.cudaFreeHost(pB)
    lib.cudaFreeHost(pX)


def test_noalloc_operator(lib, ctx):
    """mbicg_apply_D_noalloc (device pointers, a fixed scratch array) gives the
    FP32 operator of mbicg_apply_D, on two calls in a row with different
    blocks, to FP32 rounding (mbicg_apply_D reads an SU(3) field's links as two
    rows and rebuilds the third; the allocation-free call reads the caller's
    full links); sizes beyond its scratch and host pointers are refused."""
    c, U = ctx
    dims = (ctypes.c_int * 4)(*DIMS)
    dU = _device_copy(lib, U)
    try:
        for Lc, kappa, seed in ((3, 0.13, 2004), (1, 0.121, 2005)):
            psi = synth.gaussian_source(DIMS, Lc, seed=seed)
            ref = np.empty_like(psi)
            assert lib.mbicg_apply_D(c, _v(psi), _v(ref), Lc, kappa, mb.MBICG_FP32) == mb.MBICG_OK
            d_in = _device_copy(lib, psi)
            d_out = _device_copy(lib, np.full_like(psi, np.nan))
            assert lib.mbicg_apply_D_noalloc(dims, dU, d_in, d_out, Lc, kappa, None) == mb.MBICG_OK
            out = np.empty_like(psi)
            ctypes.memmove(out.ctypes.data, d_out, out.nbytes)
            V = ref.shape[0]
            d = np.linalg.norm((out - ref).reshape(V, -1), axis=1) / np.linalg.norm(ref.reshape(V, -1), axis=1)
            assert d.max() < 1e-6
            lib.cudaFree(d_in)
            lib.cudaFree(d_out)
        big = (ctypes.c_int * 4)(16, 16, 16, 16)
        assert lib.mbicg_apply_D_noalloc(big, dU, dU, dU, 12, 0.12, None) == mb.MBICG_EINVAL
        host = np.zeros_like(U)
        assert lib.mbicg_apply_D_noalloc(dims, _v(host), dU, dU, 1, 0.12, None) == mb.MBICG_EINVAL
    finally:
        lib.cudaFree(dU)


def test_memory_of_another_device_refused(lib, ctx):
    """Device memory that belongs to another device than the context's (the
    emulated runtime reports a buffer as device 1's) is refused with
    MBICG_EINVAL by the operator, the block solve and the allocation-free
    operator: their kernels would read it directly.  The same buffer reported
    as the context's device is accepted."""
    c, U = ctx
    psi = synth.gaussian_source(DIMS, 1, seed=2006)
    d_in = _device_copy(lib, psi)
    d_out = _device_copy(lib, np.zeros_like(psi))
    dU = _device_copy(lib, U)
    dims = (ctypes.c_int * 4)(*DIMS)
    p = _params(lib)
    it = ctypes.c_int(0)
    tres = np.zeros(1)
    try:
        lib.emu_set_owner(d_in, 1)
        assert lib.mbicg_apply_D(c, d_in, d_out, 1, KAPPA, mb.MBICG_FP64) == mb.MBICG_EINVAL
        assert b"another device" in lib.mbicg_last_error(c)
        assert lib.mbicg_block_solve(c, d_in, d_out, 1, KAPPA, 1e-10, ctypes.byref(p), ctypes.byref(it),
                                     tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == mb.MBICG_EINVAL
        assert lib.mbicg_apply_D_noalloc(dims, dU, d_in, d_out, 1, KAPPA, None) == mb.MBICG_EINVAL
        lib.emu_set_owner(d_in, 0)
        assert lib.mbicg_apply_D(c, d_in, d_out, 1, KAPPA, mb.MBICG_FP64) == mb.MBICG_OK
        lib.emu_set_owner(dU, 1)
        assert lib.mbicg_apply_D_noalloc(dims, dU, d_in, d_out, 1, KAPPA, None) == mb.MBICG_EINVAL
    finally:
        for d in (d_in, d_out, dU):
            lib.cudaFree(d)


def test_bounded_wait_gives_up_and_the_library_goes_on(lib, ctx, oracle_mod):
    """mbicg_selftest_bounded_wait: a wait for bytes no copy delivers gives up
    (the emulated wait ends after 2 s; on the GPU after the spin limit) and the
    kernel reports ST_TIMEOUT instead of hanging; a barrier completed by an
    arrival is waited for; afterwards a block solve, whose Gram kernel waits
    on mbarriers, still runs; the argument errors."""
    c, U = ctx
    flag = ctypes.c_int(-1)
    assert lib.mbicg_selftest_bounded_wait(0, 1000, 64, ctypes.byref(flag)) == mb.MBICG_OK and flag.value == 1
    assert lib.mbicg_selftest_bounded_wait(0, 1000, 0, ctypes.byref(flag)) == mb.MBICG_OK and flag.value == 0
    B = synth.gaussian_source(DIMS, 1, seed=2006)
    X = np.empty_like(B)
    rc, _, tres, _ = _solve(lib, c, B, X, _params(lib, prec_D=mb.MBICG_FP64))
    assert rc == mb.MBICG_OK and np.max(_residual(oracle_mod, U, B, X)) <= 1e-10
    for limit, nbytes in ((0, 16), (1 << 25, 16), (1000, -16), (1000, 8)):
        assert lib.mbicg_selftest_bounded_wait(0, limit, nbytes, ctypes.byref(flag)) == mb.MBICG_EINVAL


def test_every_cuda_source_is_emulated():
    """The emulated library is built from every CUDA source of the package."""
    sources = {f for f in os.listdir(emulation_sources.CSRC) if f.endswith(".cu")}
    assert set(emulation_sources.LIBRARY_SOURCES) == sources


def _comps(a):
    """(V, 4, 3, L) complex -> (V, L, 24) reals of each (site, rhs) spinor."""
    V, Lc = a.shape[0], a.shape[-1]
    return np.stack([a.real, a.imag], -1).reshape(V, 12, Lc, 2).transpose(0, 2, 1, 3).reshape(V, Lc, 24)


def test_fp16_operator_through_the_abi(lib, ctx, oracle_mod):
    """mbicg_apply_D with MBICG_FP16 (conversions into and out of FP16 storage
    with one scale per (site, column), the FP16 operator): kappa = 0 gives the
    input as the oracle's FP16 format represents it, bit for bit (a zero spinor
    keeps scale 0); kappa = 0.13 gives the oracle's operator on the
    FP16-represented links and input, rounded into the format, up to one FP16
    step of the output scale where the FP32 and FP64 sums round differently."""
    c, U = ctx
    psi = synth.gaussian_source(DIMS, 3, seed=2007)
    psi[3] = 0
    out = np.empty_like(psi)
    assert lib.mbicg_apply_D(c, _v(psi), _v(out), 3, 0.0, mb.MBICG_FP16) == mb.MBICG_OK
    assert np.array_equal(out, oracle.quantize_fp16(psi))
    assert lib.mbicg_apply_D(c, _v(psi), _v(out), 3, 0.13, mb.MBICG_FP16) == mb.MBICG_OK
    exp = oracle.quantize_fp16(oracle_mod.apply_D(DIMS, oracle.quantize_links_fp16(U), 0.13, oracle.quantize_fp16(psi)))
    g, e = _comps(out), _comps(exp)
    sc = np.abs(e).max(axis=2, keepdims=True)
    assert np.all(np.abs(g - e) <= 2.0 ** -10 * sc)
    assert np.mean(np.abs(g - e) > 2.0 ** -20 * sc) < 0.05


@pytest.mark.parametrize("mode,prec,tol", [(0, mb.MBICG_FP64, 1e-12), (1, mb.MBICG_FP64, 1e-12),
                                           (0, mb.MBICG_FP32, 1e-5), (1, mb.MBICG_FP32, 1e-5)])
def test_sap_precond_through_the_abi(lib, ctx, oracle_mod, mode, prec, tol):
    """mbicg_sap_precond (host pointers) against the oracle's SAP: per-column
    and block-shared MR, FP64 and FP32."""
    c, U = ctx
    eta = synth.gaussian_source(DIMS, L, seed=2008)
    out = np.empty_like(eta)
    p = _params(lib, ncycle=2, nmr=3, mr_mode=mode, prec_sap=prec)
    assert lib.mbicg_sap_precond(c, _v(eta), _v(out), L, KAPPA, ctypes.byref(p)) == mb.MBICG_OK
    ref = oracle_mod.sap(DIMS, (2, 2, 2, 2), U, KAPPA, 2, 3, eta, mr_mode=mode)
    assert np.max(np.abs(out - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec_D,dummies", [(mb.MBICG_FP64, 0), (mb.MBICG_FP32, 2)])
def test_history_and_profile_through_the_abi(lib, ctx, prec_D, dummies):
    """res_history holds the recursive residual after each iteration (one entry
    per iteration, falling to the tolerance); with profiling on, every launch
    of the solve (FP64, and mixed precision with dummy columns) is counted in
    a kernel class and timed (the emulated events read the host clock): the
    counts add up to the solve's launches, and the operator's class has its
    two launches per iteration."""
    c, _ = ctx
    lib.mbicg_set_profiling.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mbicg_get_profile.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    ncls = 10  # MBICG_K_NCLASS of include/mbicg.h
    B = synth.gaussian_source(DIMS, L, seed=2009)
    X = np.empty_like(B)
    hist = np.full(64, np.nan)
    p = _params(lib, prec_D=prec_D, dummy_rhs=dummies, dummy_seed=3)
    p.res_history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.res_history_len = len(hist)
    assert lib.mbicg_set_profiling(c, 1) == mb.MBICG_OK
    try:
        rc, iters, tres, st = _solve(lib, c, B, X, p)
        ms = np.zeros(ncls)
        n = np.zeros(ncls, dtype=np.int64)
        assert lib.mbicg_get_profile(c, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     n.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), ncls) == mb.MBICG_OK
    finally:
        lib.mbicg_set_profiling(c, 0)
    assert rc == mb.MBICG_OK and 0 < iters <= len(hist)
    h = hist[:iters]
    assert np.all(np.isfinite(h)) and np.all(np.isnan(hist[iters:]))
    assert h[-1] <= 1e-10 < h[0] and h[-1] < h[:-1].min()
    assert n.sum() == st.kernel_launches > 0 and np.all(ms >= 0) and ms.sum() > 0
    assert n[0] == 2 * iters  # MBICG_K_DSLASH
