"""The request server (include/mbicg.h, serving): columns of several requests
packed into one block solve give the same solutions as each request solved
alone, and as the oracle's solve of the same system (Algorithm 1), within
the solver's tolerance; slots of one field and of different fields solve
concurrently; compatible requests only are packed."""
import threading

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import rel_col_norm

pytestmark = pytest.mark.gpu

F1, F2 = (8, 8, 8, 16), (8, 8, 8, 8)
KAPPA, TOL = 0.125, 1e-10


def params():
    return mb.mbicg_default_params(block=(4, 4, 4, 4), ncycle=4, nmr=4, max_iter=2000)


def oracle_X(oracle_mod, dims, U, B, kappa=KAPPA):
    """The oracle's solution of A X = B (no preconditioner: X does not depend
    on it), to 1e-12."""
    r = oracle_mod.block_bicgstab(dims, U, kappa, B, 1e-12, max_iter=3000)
    assert r["status"] == 0
    return r["X"]


def solve(srv, field, B, L, kappa=KAPPA):
    rid = mb.mbicg_server_submit(srv, field, B, L, kappa, TOL)
    X = np.empty_like(B)
    st, it, tres, info = mb.mbicg_server_wait(srv, rid, X, L)
    return st, X, tres, info


def test_packed_columns_equal_solo_solves(oracle_mod):
    srv = mb.mbicg_server_create(0, 60.0)
    try:
        U1, U2 = synth.su3_links(F1, 0.5, 901), synth.su3_links(F2, 0.5, 902)
        f1 = mb.mbicg_server_add_field(srv, F1, U1, params(), 1)
        f2 = mb.mbicg_server_add_field(srv, F2, U2, params(), 1)
        B0 = synth.gaussian_source(F1, 3, seed=910)
        B1 = synth.gaussian_source(F1, 4, seed=911)
        B2 = synth.gaussian_source(F1, 5, seed=912)
        B3 = synth.gaussian_source(F2, 6, seed=913)
        # alone: one block of its own 3 columns
        st, X0, tres0, info0 = solve(srv, f1, B0, 3)
        assert st == mb.MBICG_OK and info0["batch_columns"] == 3 and max(tres0) <= TOL
        # in the mix: held, then released together; field 1's three requests
        # (3 + 4 + 5 columns, same kappa) form one block of 12, field 2 runs beside it
        mb.mbicg_server_hold(srv, True)
        ids = [(mb.mbicg_server_submit(srv, f1, B0, 3, KAPPA, TOL), B0, 3),
               (mb.mbicg_server_submit(srv, f1, B1, 4, KAPPA, TOL), B1, 4),
               (mb.mbicg_server_submit(srv, f1, B2, 5, KAPPA, TOL), B2, 5),
               (mb.mbicg_server_submit(srv, f2, B3, 6, KAPPA, TOL), B3, 6)]
        mb.mbicg_server_hold(srv, False)
        res = []
        for rid, B, L in ids:
            X = np.empty_like(B)
            st, it, tres, info = mb.mbicg_server_wait(srv, rid, X, L)
            assert st == mb.MBICG_OK and max(tres) <= TOL
            res.append((X, info))
        assert [r[1]["batch_columns"] for r in res] == [12, 12, 12, 6]
        # the same solution alone and in the mix: both within tol of A^-1 b,
        # so they differ by at most cond * tol; 1e-7 is the stated bound
        assert rel_col_norm(res[0][0], X0) < 1e-7
        # and every request's columns against the oracle's solve of its system
        assert rel_col_norm(X0, oracle_X(oracle_mod, F1, U1, B0)) < 1e-7
        assert rel_col_norm(res[0][0], oracle_X(oracle_mod, F1, U1, B0)) < 1e-7
        assert rel_col_norm(res[1][0], oracle_X(oracle_mod, F1, U1, B1)) < 1e-7
        assert rel_col_norm(res[2][0], oracle_X(oracle_mod, F1, U1, B2)) < 1e-7
        assert rel_col_norm(res[3][0], oracle_X(oracle_mod, F2, U2, B3)) < 1e-7
        # field 2's solve overlapped field 1's block
        a, b = res[0][1], res[3][1]
        assert a["start_ms"] < b["done_ms"] and b["start_ms"] < a["done_ms"]
        s = mb.mbicg_server_stats(srv)
        assert s["solves"] == 3 and s["max_columns"] == 12 and s["slots"] == 2
    finally:
        mb.mbicg_server_destroy(srv)


def test_two_slots_of_one_field_overlap_and_kappas_are_not_mixed(oracle_mod):
    srv = mb.mbicg_server_create(0, 60.0)
    try:
        U = synth.su3_links(F1, 0.5, 903)
        f = mb.mbicg_server_add_field(srv, F1, U, params(), 2)
        B = [synth.gaussian_source(F1, 6, seed=920 + i) for i in range(4)]
        mb.mbicg_server_hold(srv, True)
        ids = [mb.mbicg_server_submit(srv, f, B[0], 6, 0.12, TOL), mb.mbicg_server_submit(srv, f, B[1], 6, 0.125, TOL),
               mb.mbicg_server_submit(srv, f, B[2], 6, 0.12, TOL), mb.mbicg_server_submit(srv, f, B[3], 6, 0.125, TOL)]
        mb.mbicg_server_hold(srv, False)
        infos = []
        for rid, b, kappa in zip(ids, B, (0.12, 0.125, 0.12, 0.125)):
            X = np.empty_like(b)
            st, it, tres, info = mb.mbicg_server_wait(srv, rid, X, 6)
            assert st == mb.MBICG_OK and max(tres) <= TOL
            assert rel_col_norm(X, oracle_X(oracle_mod, F1, U, b, kappa)) < 1e-7
            infos.append(info)
        # requests 0 and 2 (kappa 0.12) share a block, 1 and 3 (0.125) another
        assert [i["batch_columns"] for i in infos] == [12, 12, 12, 12]
        assert infos[0]["start_ms"] == infos[2]["start_ms"] and infos[1]["start_ms"] == infos[3]["start_ms"]
        assert infos[0]["start_ms"] < infos[1]["done_ms"] and infos[1]["start_ms"] < infos[0]["done_ms"]
    finally:
        mb.mbicg_server_destroy(srv)


def test_concurrent_submitters_and_bad_requests(oracle_mod):
    srv = mb.mbicg_server_create(0, 60.0)
    try:
        f = mb.mbicg_server_add_field(srv, F2, synth.su3_links(F2, 0.5, 904), params(), 2)
        B = synth.gaussian_source(F2, 2, seed=930)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_server_submit(srv, 7, B, 2, KAPPA, TOL)       # unknown field
        with pytest.raises(mb.MbicgError):
            mb.mbicg_server_submit(srv, f, synth.gaussian_source(F2, 13, seed=1), 13, KAPPA, TOL)
        with pytest.raises(mb.MbicgError):
            mb.mbicg_server_submit(srv, f, B, 2, KAPPA, 0.0)
        out = {}

        def client(i):
            b = synth.gaussian_source(F2, 1 + i % 3, seed=940 + i)
            out[i] = (b, solve(srv, f, b, b.shape[-1]))

        th = [threading.Thread(target=client, args=(i,)) for i in range(8)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        U = synth.su3_links(F2, 0.5, 904)
        for i, (b, (st, X, tres, info)) in out.items():
            assert st == mb.MBICG_OK and max(tres) <= TOL
            assert rel_col_norm(X, oracle_X(oracle_mod, F2, U, b)) < 1e-7
    finally:
        mb.mbicg_server_destroy(srv)


def solve_bytes(V, L):
    """The server's estimate of a block solve's workspace (FP32 Krylov
    vectors and SAP storage, include/mbicg.h): 12 V L (3*16 + 7*8 + 3*8 +
    3*16) bytes, 5 % margin and 8 MiB."""
    return 1.05 * 12 * V * L * (3 * 16 + 7 * 8 + 3 * 8 + 3 * 16) + (8 << 20)


def test_admission_by_hbm_footprint(oracle_mod):
    """Work is admitted by device-memory footprint as it arrives: with a
    budget that holds the links of two slots and the workspace of only one
    12-column block solve, the two slots never solve at the same time (the
    second waits for memory), every request is solved, and the server never
    holds more than its budget; a request whose block can never fit is
    refused at submit; a budget below one slot's links refuses the field."""
    U = synth.su3_links(F2, 0.5, 905)
    V = int(np.prod(F2))
    srv = mb.mbicg_server_create(0, 1e-3)
    try:
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_server_add_field(srv, F2, U, params(), 3)
        assert e.value.status == mb.MBICG_ENOMEM
    finally:
        mb.mbicg_server_destroy(srv)
    links = 2 * (V * 1152 + (1 << 22))  # FP64, FP32, FP16-row and FP32-row links per slot
    budget = links + 1.5 * solve_bytes(V, 12)
    srv = mb.mbicg_server_create(0, budget / 1e9)
    try:
        f = mb.mbicg_server_add_field(srv, F2, U, params(), 2)
        assert mb.mbicg_server_stats(srv)["slots"] == 2
        mb.mbicg_server_hold(srv, True)
        Bs = [synth.gaussian_source(F2, 12, seed=950 + i) for i in range(4)]
        kappas = (0.12, 0.125, 0.12, 0.125)  # no two of them pack together (12 columns each)
        ids = [mb.mbicg_server_submit(srv, f, B, 12, k, TOL) for B, k in zip(Bs, kappas)]
        mb.mbicg_server_hold(srv, False)
        infos = []
        for rid, B, k in zip(ids, Bs, kappas):
            X = np.empty_like(B)
            st, it, tres, info = mb.mbicg_server_wait(srv, rid, X, 12)
            assert st == mb.MBICG_OK and max(tres) <= TOL
            assert rel_col_norm(X, oracle_X(oracle_mod, F2, U, B, k)) < 1e-7
            infos.append(info)
        spans = sorted((i["start_ms"], i["done_ms"]) for i in infos)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert b0 >= a1  # one 12-column solve at a time
        mem = mb.mbicg_server_memory(srv)
        assert mem["memory_waits"] >= 1
        assert mem["used_gb"] * 1e9 <= budget
        # a block that could never fit is refused at submit
        srv2 = mb.mbicg_server_create(0, (links + 0.5 * solve_bytes(V, 12)) / 1e9)
        try:
            f2 = mb.mbicg_server_add_field(srv2, F2, U, params(), 2)
            with pytest.raises(mb.MbicgError) as e:
                mb.mbicg_server_submit(srv2, f2, Bs[0], 12, 0.12, TOL)
            assert e.value.status == mb.MBICG_ENOMEM
            # two columns fit: admitted and solved
            b2 = np.ascontiguousarray(Bs[0][..., :2])
            st, X2, tres2, _ = solve(srv2, f2, b2, 2, 0.12)
            assert st == mb.MBICG_OK and max(tres2) <= TOL
        finally:
            mb.mbicg_server_destroy(srv2)
    finally:
        mb.mbicg_server_destroy(srv)
