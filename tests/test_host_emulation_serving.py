"""The request server (include/mbicg.h, serving) on the CPU through the C ABI
of the emulated library (tests/emulated_library.py): its slots are host
threads that run the library's own block solves on the emulator.  Columns of
several requests packed into one block solve give the solutions of each
request solved alone, within the solver's tolerance; requests of different
kappas are not packed together; requests submitted and waited for from
several host threads at once get their own solutions (checked with the
oracle's operator); the argument errors."""
import ctypes
import threading

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb  # the ctypes structures only; no library is loaded
import synth

F1, F2, BLOCK = (4, 4, 4, 4), (4, 4, 4, 8), (2, 2, 2, 2)
KAPPA, TOL = 0.12, 1e-10


def _v(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.fixture(scope="module")
def lib(emulated_library):
    return emulated_library


def _params(lib, **kw):
    p = mb.mbicg_params()
    lib.mbicg_default_params(ctypes.byref(p))
    p.block = (ctypes.c_int * 4)(*BLOCK)
    p.max_iter = 2000
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Server:
    def __init__(self, lib):
        self.lib = lib
        self.s = ctypes.c_void_p()
        assert lib.mbicg_server_create(ctypes.byref(self.s), 0, 1.0) == mb.MBICG_OK

    def add_field(self, dims, U, slots):
        fid = ctypes.c_int(-1)
        p = _params(self.lib)
        assert self.lib.mbicg_server_add_field(self.s, (ctypes.c_int * 4)(*dims), _v(U), ctypes.byref(p), slots,
                                               ctypes.byref(fid)) == mb.MBICG_OK
        return fid.value

    def submit(self, fid, B, kappa=KAPPA, tol=TOL, L=None):
        rid = ctypes.c_longlong(-1)
        rc = self.lib.mbicg_server_submit(self.s, fid, _v(B), B.shape[3] if L is None else L, kappa, tol,
                                          ctypes.byref(rid))
        return rc, rid.value

    def wait(self, rid, B):
        X = np.empty_like(B)
        it = ctypes.c_int(0)
        tres = np.zeros(B.shape[3])
        info = mb.mbicg_request_info()
        rc = self.lib.mbicg_server_wait(self.s, rid, _v(X), ctypes.byref(it),
                                        tres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(info))
        return rc, X, tres, info

    def stats(self):
        v = [ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_int(0)]
        assert self.lib.mbicg_server_stats(self.s, *[ctypes.byref(x) for x in v]) == mb.MBICG_OK
        return [x.value for x in v]

    def close(self):
        self.lib.mbicg_server_destroy(self.s)


def _rel_col(a, b):
    n = a.shape[3]
    return float(np.max(np.linalg.norm((a - b).reshape(-1, n), axis=0) / np.linalg.norm(b.reshape(-1, n), axis=0)))


def test_packed_columns_equal_solo_solves(lib):
    srv = Server(lib)
    try:
        f1 = srv.add_field(F1, synth.su3_links(F1, 0.5, seed=1300), 1)
        f2 = srv.add_field(F2, synth.su3_links(F2, 0.5, seed=1301), 1)
        B = [synth.gaussian_source(F1, L, seed=1310 + L) for L in (1, 2, 3)]
        B2 = synth.gaussian_source(F2, 2, seed=1314)
        rc, rid = srv.submit(f1, B[0])
        rc, X0, tres0, info0 = srv.wait(rid, B[0])
        assert rc == mb.MBICG_OK and info0.batch_columns == 1 and tres0.max() <= TOL
        # held, then released: field 1's three requests form one block of 6
        # columns, field 2's request runs in its own slot
        assert lib.mbicg_server_hold(srv.s, 1) == mb.MBICG_OK
        ids = [srv.submit(f1, b)[1] for b in B] + [srv.submit(f2, B2)[1]]
        assert lib.mbicg_server_hold(srv.s, 0) == mb.MBICG_OK
        res = [srv.wait(rid, b) for rid, b in zip(ids, B + [B2])]
        assert all(r[0] == mb.MBICG_OK and r[2].max() <= TOL for r in res)
        assert [r[3].batch_columns for r in res] == [6, 6, 6, 2]
        # the same column alone and in the block: both within tol of A^-1 b
        assert _rel_col(res[0][1], X0) < 1e-7
        solves, columns, widest, slots = srv.stats()
        assert (solves, columns, widest, slots) == (3, 9, 6, 2)
    finally:
        srv.close()


def test_kappas_are_not_mixed(lib):
    srv = Server(lib)
    try:
        f = srv.add_field(F1, synth.su3_links(F1, 0.5, seed=1302), 2)
        B = [synth.gaussian_source(F1, 2, seed=1320 + i) for i in range(4)]
        assert lib.mbicg_server_hold(srv.s, 1) == mb.MBICG_OK
        ids = [srv.submit(f, b, kappa=k)[1] for b, k in zip(B, (0.12, 0.125, 0.12, 0.125))]
        assert lib.mbicg_server_hold(srv.s, 0) == mb.MBICG_OK
        res = [srv.wait(rid, b) for rid, b in zip(ids, B)]
        assert all(r[0] == mb.MBICG_OK for r in res)
        assert [r[3].batch_columns for r in res] == [4, 4, 4, 4]
        assert srv.stats()[:3] == [2, 8, 4]
    finally:
        srv.close()


def test_concurrent_submitters(lib, oracle_mod):
    srv = Server(lib)
    U = synth.su3_links(F1, 0.5, seed=1303)
    try:
        f = srv.add_field(F1, U, 2)
        B = [synth.gaussian_source(F1, 1 + i % 3, seed=1330 + i) for i in range(6)]
        out = [None] * len(B)

        def client(i):
            rc, rid = srv.submit(f, B[i])
            out[i] = (rc,) + srv.wait(rid, B[i])

        threads = [threading.Thread(target=client, args=(i,)) for i in range(len(B))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for b, (rc_submit, rc, X, tres, info) in zip(B, out):
            assert rc_submit == mb.MBICG_OK and rc == mb.MBICG_OK and tres.max() <= TOL
            R = b - oracle_mod.apply_D(F1, U, KAPPA, X)
            n = b.shape[3]
            rel = np.linalg.norm(R.reshape(-1, n), axis=0) / np.linalg.norm(b.reshape(-1, n), axis=0)
            assert rel.max() <= 1e-9
        assert srv.stats()[1] == sum(b.shape[3] for b in B)
    finally:
        srv.close()


def test_fields_added_while_slots_solve(lib, oracle_mod):
    """Fields added while another field's block solves run (the server's list
    of fields grows under the running slots): every request, before and after,
    is solved on its own field (residual with the oracle's operator)."""
    srv = Server(lib)
    U1 = synth.su3_links(F1, 0.5, seed=1305)
    try:
        f1 = srv.add_field(F1, U1, 2)
        B = [synth.gaussian_source(F1, 3, seed=1350 + i) for i in range(2)]
        ids = [srv.submit(f1, b)[1] for b in B]
        extra = []
        for k, dims in enumerate((F2, (4, 4, 8, 4), (8, 4, 4, 4))):
            U = synth.su3_links(dims, 0.5, seed=1306 + k)
            extra.append((dims, U, srv.add_field(dims, U, 1)))
        checks = [(rid, b, F1, U1) for rid, b in zip(ids, B)]
        for dims, U, f in extra:
            b = synth.gaussian_source(dims, 2, seed=1360 + f)
            checks.append((srv.submit(f, b)[1], b, dims, U))
        for rid, b, dims, U in checks:
            rc, X, tres, info = srv.wait(rid, b)
            assert rc == mb.MBICG_OK and tres.max() <= TOL
            R = b - oracle_mod.apply_D(dims, U, KAPPA, X)
            n = b.shape[3]
            rel = np.linalg.norm(R.reshape(-1, n), axis=0) / np.linalg.norm(b.reshape(-1, n), axis=0)
            assert rel.max() <= 1e-9
        assert srv.stats()[3] == 5
    finally:
        srv.close()


def test_one_wait_per_request(lib):
    """Two host threads waiting for the same request: one gets the solution,
    the other MBICG_EINVAL (whether it came while the first waited or after it
    returned); a wait after that is refused too."""
    srv = Server(lib)
    try:
        f = srv.add_field(F1, synth.su3_links(F1, 0.5, seed=1307), 1)
        B = synth.gaussian_source(F1, 2, seed=1370)
        rc, rid = srv.submit(f, B)
        assert rc == mb.MBICG_OK
        out = [None, None]

        def waiter(i):
            out[i] = srv.wait(rid, B)

        threads = [threading.Thread(target=waiter, args=(i,)) for i in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        codes = sorted(o[0] for o in out)
        assert codes == sorted([mb.MBICG_OK, mb.MBICG_EINVAL])
        good = next(o for o in out if o[0] == mb.MBICG_OK)
        assert good[2].max() <= TOL
        assert srv.wait(rid, B)[0] == mb.MBICG_EINVAL
    finally:
        srv.close()


def _solve_bytes(V, L):
    """The server's estimate of one block solve's workspace with the default
    parameters (FP32 Krylov vectors and SAP storage) and the packing buffers:
    12 V L (3*16 + 7*8 + 3*8 + 3*16) bytes, 5 % margin and 8 MiB."""
    return 1.05 * 12 * V * L * (3 * 16 + 7 * 8 + 3 * 8 + 3 * 16) + (8 << 20)


def test_admission_by_memory_budget(lib, oracle_mod):
    """Two slots and a budget for their links and one 4-column block solve:
    the slots never solve at once (the second waits for memory, idle slots
    give their workspaces back), every request is solved on its own (kappas
    differ, so nothing packs), and the memory held stays within the budget."""
    V = int(np.prod(F1))
    links = 2 * (V * 1152 + (1 << 22))
    budget = links + 1.5 * _solve_bytes(V, 4)
    s = ctypes.c_void_p()
    assert lib.mbicg_server_create(ctypes.byref(s), 0, budget / 1e9) == mb.MBICG_OK
    srv = Server.__new__(Server)
    srv.lib, srv.s = lib, s
    U = synth.su3_links(F1, 0.5, seed=1308)
    try:
        f = srv.add_field(F1, U, 2)
        assert srv.stats()[3] == 2
        kappas = (0.12, 0.121, 0.122, 0.123)  # all different: no two requests pack together
        B = [synth.gaussian_source(F1, 4, seed=1380 + i) for i in range(4)]
        assert lib.mbicg_server_hold(s, 1) == mb.MBICG_OK
        ids = [srv.submit(f, b, kappa=k)[1] for b, k in zip(B, kappas)]
        assert lib.mbicg_server_hold(s, 0) == mb.MBICG_OK
        spans = []
        for rid, b, k in zip(ids, B, kappas):
            rc, X, tres, info = srv.wait(rid, b)
            assert rc == mb.MBICG_OK and tres.max() <= TOL
            R = b - oracle_mod.apply_D(F1, U, k, X)
            rel = np.linalg.norm(R.reshape(-1, 4), axis=0) / np.linalg.norm(b.reshape(-1, 4), axis=0)
            assert rel.max() <= 1e-9
            spans.append((info.start_ms, info.done_ms))
        spans.sort()
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert b0 >= a1  # one block solve at a time
        used, cap, waits = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        assert lib.mbicg_server_memory(s, ctypes.byref(used), ctypes.byref(cap), ctypes.byref(waits)) == 0
        assert waits.value >= 1 and used.value * 1e9 <= budget
    finally:
        srv.close()


def test_request_that_can_no_longer_fit_ends_with_enomem(lib):
    """A request admitted at submit (its block fits beside the links held
    then), after which a second field's links take the budget: with nothing
    running and no idle workspace to release, it can never be admitted and its
    wait returns MBICG_ENOMEM instead of waiting forever; a smaller request
    that still fits is solved afterwards."""
    V1, V2 = int(np.prod(F1)), int(np.prod(F2))
    links = (V1 * 1152 + (1 << 22)) + (V2 * 1152 + (1 << 22))
    budget = links + _solve_bytes(V1, 4) - 1e3
    s = ctypes.c_void_p()
    assert lib.mbicg_server_create(ctypes.byref(s), 0, budget / 1e9) == mb.MBICG_OK
    srv = Server.__new__(Server)
    srv.lib, srv.s = lib, s
    try:
        f1 = srv.add_field(F1, synth.su3_links(F1, 0.5, seed=1309), 1)
        B4 = synth.gaussian_source(F1, 4, seed=1390)
        assert lib.mbicg_server_hold(s, 1) == mb.MBICG_OK
        rc, rid = srv.submit(f1, B4)
        assert rc == mb.MBICG_OK
        srv.add_field(F2, synth.su3_links(F2, 0.5, seed=1310), 1)
        assert lib.mbicg_server_hold(s, 0) == mb.MBICG_OK
        assert srv.wait(rid, B4)[0] == mb.MBICG_ENOMEM
        B1 = synth.gaussian_source(F1, 1, seed=1391)
        rc, rid = srv.submit(f1, B1)
        assert rc == mb.MBICG_OK
        rc, X, tres, info = srv.wait(rid, B1)
        assert rc == mb.MBICG_OK and tres.max() <= TOL
    finally:
        srv.close()


def test_server_argument_errors(lib):
    srv = Server(lib)
    try:
        f = srv.add_field(F1, synth.su3_links(F1, 0.5, seed=1304), 1)
        B = synth.gaussian_source(F1, 1, seed=1340)
        assert srv.submit(f + 7, B)[0] == mb.MBICG_EINVAL
        assert srv.submit(f, B, L=0)[0] == mb.MBICG_EINVAL
        assert srv.submit(f, B, L=13)[0] == mb.MBICG_EINVAL
        assert srv.submit(f, B, tol=0.0)[0] == mb.MBICG_EINVAL
    finally:
        srv.close()
