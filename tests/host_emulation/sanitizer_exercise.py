"""Drives the emulated library through its C ABI in a build with sanitizers:
AddressSanitizer with UndefinedBehaviorSanitizer ("address") or
ThreadSanitizer ("thread").  Started by
tests/test_host_emulation_sanitizers.py as a child process with the
sanitizer's runtime preloaded; arguments: the library's path and the
sanitizer.  Every call must return MBICG_OK and the sanitizers must report
nothing; the numbers themselves are checked against the oracle by the other
emulation tests, here only for being finite and converged."""
import ctypes
import os
import sys
import threading
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]

import numpy as np  # noqa: E402

import emulated_library  # noqa: E402
import paper_1104_0737_gb300 as mb  # noqa: E402  (the ctypes structures only)
import synth  # noqa: E402

KAPPA = 0.12
T0 = time.perf_counter()


def _v(a):
    return ctypes.c_void_p(a.ctypes.data)


class Ctx:
    def __init__(self, lib, dims, seed):
        self.lib, self.dims = lib, dims
        self.c = ctypes.c_void_p()
        assert lib.mbicg_create(ctypes.byref(self.c), (ctypes.c_int * 4)(*dims), 0, None) == mb.MBICG_OK
        self.U = synth.su3_links(dims, 0.5, seed=seed)
        assert lib.mbicg_load_gauge(self.c, _v(self.U)) == mb.MBICG_OK

    def close(self):
        self.lib.mbicg_destroy(self.c)

    def params(self, block, **kw):
        p = mb.mbicg_params()
        self.lib.mbicg_default_params(ctypes.byref(p))
        p.block = (ctypes.c_int * 4)(*block)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def ok(self, rc, what):
        assert rc == mb.MBICG_OK, f"{what}: {rc} {self.lib.mbicg_last_error(self.c)}"
        print(f"ok {what} ({time.perf_counter() - T0:.1f} s)", flush=True)

    def apply_D(self, L, prec):
        psi = synth.gaussian_source(self.dims, L, seed=10 + L)
        out = np.empty_like(psi)
        self.ok(self.lib.mbicg_apply_D(self.c, _v(psi), _v(out), L, KAPPA, prec), f"apply_D L={L} prec={prec}")
        assert np.isfinite(out).all()

    def sap(self, L, block, **kw):
        eta = synth.gaussian_source(self.dims, L, seed=20 + L)
        out = np.empty_like(eta)
        p = self.params(block, **kw)
        self.ok(self.lib.mbicg_sap_precond(self.c, _v(eta), _v(out), L, KAPPA, ctypes.byref(p)),
                f"sap {self.dims} L={L} {kw}")
        assert np.isfinite(out).all()

    def solve(self, L, block, tol=1e-9, X=None, **kw):
        B = synth.gaussian_source(self.dims, L, seed=30 + L)
        X = np.empty_like(B) if X is None else X
        p = self.params(block, **kw)
        it = ctypes.c_int(0)
        tres = np.zeros(L)
        self.ok(self.lib.mbicg_block_solve(self.c, _v(B), _v(X), L, KAPPA, tol, ctypes.byref(p), ctypes.byref(it),
                                           tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                f"block_solve {self.dims} L={L} {kw}")
        assert tres.max() <= tol, tres
        return X


def check_sanitizer(lib):
    """Both sanitizers are live, and an emulated device buffer ends exactly at
    its size: the byte after it is poisoned, its last byte is not."""
    lib["__ubsan_handle_type_mismatch_v1_abort"]  # the alignment check's handler
    is_poisoned = ctypes.CDLL(None).__asan_address_is_poisoned
    is_poisoned.argtypes = [ctypes.c_void_p]
    p = ctypes.c_void_p()
    assert lib.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(1000)) == 0
    assert is_poisoned(p.value + 999) == 0 and is_poisoned(p.value + 1000) == 1
    lib.cudaFree(p)
    print("ok sanitizer", flush=True)


def main(so, sanitizer):
    lib = emulated_library.load(so)
    if sanitizer == "address":
        check_sanitizer(lib)
    else:
        lib["__tsan_func_entry"]  # the library is instrumented for ThreadSanitizer
        print("ok sanitizer", flush=True)
    small = Ctx(lib, (4, 4, 4, 4), seed=1)
    b2 = (2, 2, 2, 2)
    for L in (1, 3):
        for prec in (mb.MBICG_FP64, mb.MBICG_FP32, mb.MBICG_FP16):
            small.apply_D(L, prec)
    # the allocation-free operator on emulated device buffers
    U, psi = small.U, synth.gaussian_source(small.dims, 3, seed=60)
    bufs = []
    for a in (U, psi, psi):
        p = ctypes.c_void_p()
        assert lib.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(a.nbytes)) == 0
        ctypes.memmove(p, a.ctypes.data, a.nbytes)
        bufs.append(p)
    small.ok(lib.mbicg_apply_D_noalloc((ctypes.c_int * 4)(*small.dims), bufs[0], bufs[1], bufs[2], 3, KAPPA, None),
             "apply_D_noalloc L=3")
    for p in bufs:
        lib.cudaFree(p)
    # page-locked host blocks: staged by the mapped-host copy kernel
    nbytes = int(np.prod(small.dims)) * 12 * 3 * 16
    hb = [ctypes.c_void_p() for _ in range(2)]
    for p in hb:
        assert lib.cudaMallocHost(ctypes.byref(p), ctypes.c_size_t(nbytes)) == 0
    ctypes.memmove(hb[0], psi.ctypes.data, nbytes)
    small.ok(lib.mbicg_apply_D(small.c, hb[0], hb[1], 3, KAPPA, mb.MBICG_FP32), "apply_D from page-locked memory")
    for p in hb:
        lib.cudaFreeHost(p)
    for fused in ("1", "0"):
        os.environ["MBICG_SAP_FUSED"] = fused
        for mode in (mb.MBICG_MR_COLUMN, mb.MBICG_MR_BLOCK):
            for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
                small.sap(3, b2, ncycle=1, nmr=2, mr_mode=mode, prec_sap=prec)
    os.environ.pop("MBICG_SAP_FUSED")
    small.solve(2, b2, prec_D=mb.MBICG_FP64)
    X = small.solve(3, b2, prec_D=mb.MBICG_FP32, dummy_rhs=2, dummy_seed=5)
    small.solve(3, b2, X=X, use_x0=1)
    # SSOR domain solves, the clover term and its Jacobi preconditioning (Sec. 2.2)
    for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
        small.sap(3, b2, ncycle=1, prec_sap=prec, domain_solver=1, nssor=2)
    lib.mbicg_load_clover.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.mbicg_apply_clover.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_int]
    small.ok(lib.mbicg_load_clover(small.c, 1.3), "load_clover")
    psi = synth.gaussian_source(small.dims, 3, seed=40)
    out = np.empty_like(psi)
    for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
        for jacobi in (0, 1):
            small.ok(lib.mbicg_apply_clover(small.c, _v(psi), _v(out), 3, KAPPA, prec, jacobi),
                     f"apply_clover prec={prec} jacobi={jacobi}")
            assert np.isfinite(out).all()
    for solver in (0, 1):
        for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
            small.sap(3, b2, ncycle=1, nmr=2, mr_mode=mb.MBICG_MR_COLUMN, prec_sap=prec, clover=1,
                      domain_solver=solver)
        small.solve(2, b2, clover=1, domain_solver=solver)
    small.close()

    # every launch configuration of the operator the autotuner times (CTA
    # sizes, lexicographic and time-slab order), on a lattice where the slabs apply
    os.environ["MBICG_AUTOTUNE"] = "1"
    tuned = Ctx(lib, (4, 4, 4, 8), seed=3)
    tuned.solve(2, (2, 2, 2, 4), tol=1e-6)
    tuned.close()
    os.environ.pop("MBICG_AUTOTUNE")

    # the request server: two slots of one field, four clients on host threads
    srv = ctypes.c_void_p()
    assert lib.mbicg_server_create(ctypes.byref(srv), 0, 1.0) == mb.MBICG_OK
    dims = (4, 4, 4, 4)
    fid = ctypes.c_int(-1)
    p = mb.mbicg_params()
    lib.mbicg_default_params(ctypes.byref(p))
    p.block = (ctypes.c_int * 4)(2, 2, 2, 2)
    U = synth.su3_links(dims, 0.5, seed=4)
    assert lib.mbicg_server_add_field(srv, (ctypes.c_int * 4)(*dims), _v(U), ctypes.byref(p), 2,
                                      ctypes.byref(fid)) == mb.MBICG_OK
    results = [None] * 4

    def client(i):
        B = synth.gaussian_source(dims, 1 + i % 2, seed=50 + i)
        rid = ctypes.c_longlong(-1)
        rc = lib.mbicg_server_submit(srv, fid.value, _v(B), B.shape[3], KAPPA, 1e-4, ctypes.byref(rid))
        X = np.empty_like(B)
        tres = np.zeros(B.shape[3])
        rc2 = lib.mbicg_server_wait(srv, rid.value, _v(X), None, tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    None)
        results[i] = (rc, rc2, float(tres.max()))

    clients = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for t in clients:
        t.start()
    # two more fields added while the clients' block solves run (the server's
    # list of fields grows under the running slots), each then given a request
    more = []
    for k, d in enumerate(((4, 4, 4, 8), (4, 4, 8, 4))):
        f2 = ctypes.c_int(-1)
        U2 = synth.su3_links(d, 0.5, seed=5 + k)
        assert lib.mbicg_server_add_field(srv, (ctypes.c_int * 4)(*d), _v(U2), ctypes.byref(p), 1,
                                          ctypes.byref(f2)) == mb.MBICG_OK
        more.append((d, f2.value))
    for t in clients:
        t.join()
    for d, f2 in more:
        B = synth.gaussian_source(d, 2, seed=60 + f2)
        rid = ctypes.c_longlong(-1)
        assert lib.mbicg_server_submit(srv, f2, _v(B), 2, KAPPA, 1e-4, ctypes.byref(rid)) == mb.MBICG_OK
        X = np.empty_like(B)
        tres = np.zeros(2)
        rc2 = lib.mbicg_server_wait(srv, rid.value, _v(X), None, tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    None)
        results.append((mb.MBICG_OK, rc2, float(tres.max())))
    lib.mbicg_server_destroy(srv)
    assert all(r[0] == mb.MBICG_OK and r[1] == mb.MBICG_OK and r[2] <= 1e-4 for r in results), results

    # admission by memory: two slots, a budget for their links and one
    # 2-column block solve; two requests of different kappas, so the second
    # slot waits for memory and releases the idle slot's workspace
    V = 4 ** 4
    budget = 2 * (V * 1152 + (1 << 22)) + 1.5 * (1.05 * 12 * V * 2 * 176 + (8 << 20))
    srv = ctypes.c_void_p()
    assert lib.mbicg_server_create(ctypes.byref(srv), 0, budget / 1e9) == mb.MBICG_OK
    fid = ctypes.c_int(-1)
    assert lib.mbicg_server_add_field(srv, (ctypes.c_int * 4)(*dims), _v(U), ctypes.byref(p), 2,
                                      ctypes.byref(fid)) == mb.MBICG_OK
    assert lib.mbicg_server_hold(srv, 1) == mb.MBICG_OK
    reqs = []
    for k, kappa in enumerate((0.12, 0.125, 0.12)):
        B = synth.gaussian_source(dims, 2, seed=70 + k)
        rid = ctypes.c_longlong(-1)
        assert lib.mbicg_server_submit(srv, fid.value, _v(B), 2, kappa, 1e-4, ctypes.byref(rid)) == mb.MBICG_OK
        reqs.append((rid.value, B))
    assert lib.mbicg_server_hold(srv, 0) == mb.MBICG_OK
    for rid, B in reqs:
        X = np.empty_like(B)
        tres = np.zeros(2)
        rc2 = lib.mbicg_server_wait(srv, rid, _v(X), None, tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    None)
        assert rc2 == mb.MBICG_OK and tres.max() <= 1e-4, (rc2, tres)
    lib.mbicg_server_destroy(srv)

    # a request that a field added after its submission made unadmissible
    # ends with MBICG_ENOMEM (no solve runs, no idle workspace to release)
    d2 = (4, 4, 4, 8)
    budget = (V * 1152 + (1 << 22)) + (2 * V * 1152 + (1 << 22)) + (1.05 * 12 * V * 2 * 176 + (8 << 20)) - 1e3
    srv = ctypes.c_void_p()
    assert lib.mbicg_server_create(ctypes.byref(srv), 0, budget / 1e9) == mb.MBICG_OK
    assert lib.mbicg_server_add_field(srv, (ctypes.c_int * 4)(*dims), _v(U), ctypes.byref(p), 1,
                                      ctypes.byref(fid)) == mb.MBICG_OK
    assert lib.mbicg_server_hold(srv, 1) == mb.MBICG_OK
    B = synth.gaussian_source(dims, 2, seed=80)
    rid = ctypes.c_longlong(-1)
    assert lib.mbicg_server_submit(srv, fid.value, _v(B), 2, KAPPA, 1e-4, ctypes.byref(rid)) == mb.MBICG_OK
    f2 = ctypes.c_int(-1)
    U2 = synth.su3_links(d2, 0.5, seed=8)
    assert lib.mbicg_server_add_field(srv, (ctypes.c_int * 4)(*d2), _v(U2), ctypes.byref(p), 1,
                                      ctypes.byref(f2)) == mb.MBICG_OK
    assert lib.mbicg_server_hold(srv, 0) == mb.MBICG_OK
    X = np.empty_like(B)
    assert lib.mbicg_server_wait(srv, rid.value, _v(X), None, None, None) == mb.MBICG_ENOMEM
    lib.mbicg_server_destroy(srv)
    print(f"ok server ({time.perf_counter() - T0:.1f} s)", flush=True)

    # the 8-CTA cluster sweep over 4^4 domains, and an iteration or two of a
    # block solve on it (the frozen step lengths recorded, then replayed)
    big = Ctx(lib, (8, 8, 8, 8), seed=2)
    b4 = (4, 4, 4, 4)
    big.sap(1, b4, ncycle=1, nmr=2, mr_mode=mb.MBICG_MR_COLUMN)
    if sanitizer == "address":  # the same kernels as the sweep above, at the cost of a solve
        big.solve(1, b4, tol=1e-1, ncycle=1, nmr=2)
    big.close()
    print("done", flush=True)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2] if len(sys.argv) > 2 else "address")
