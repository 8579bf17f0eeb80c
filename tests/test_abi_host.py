"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/mbicg.h declares, its ctypes
structures match the C layout, and it fails cleanly without a device."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1104_0737_gb300 as mb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mbicg.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(mbicg_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_function():
    lib = mb.load_library()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    # the binding exposes the same names
    for n in names:
        assert hasattr(mb, n), n


def test_ctypes_structs_match_c_layout(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('''
#include <stddef.h>
#include <stdio.h>
#include "mbicg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mbicg_params), offsetof(mbicg_params, delta_ru),
         offsetof(mbicg_params, res_history), offsetof(mbicg_params, res_history_len),
         sizeof(mbicg_stats), offsetof(mbicg_stats, true_res_max),
         sizeof(mbicg_request_info), offsetof(mbicg_request_info, batch_columns),
         offsetof(mbicg_stats, graph_iterations), offsetof(mbicg_stats, precision_fallbacks),
         offsetof(mbicg_params, dummy_rhs), offsetof(mbicg_params, dummy_seed), offsetof(mbicg_params, clover),
         offsetof(mbicg_params, domain_solver), offsetof(mbicg_params, nssor), offsetof(mbicg_params, ssor_omega),
         offsetof(mbicg_stats, host_syncs));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(mb.mbicg_params), mb.mbicg_params.delta_ru.offset,
            mb.mbicg_params.res_history.offset, mb.mbicg_params.res_history_len.offset,
            ctypes.sizeof(mb.mbicg_stats), mb.mbicg_stats.true_res_max.offset,
            ctypes.sizeof(mb.mbicg_request_info), mb.mbicg_request_info.batch_columns.offset,
            mb.mbicg_stats.graph_iterations.offset, mb.mbicg_stats.precision_fallbacks.offset,
            mb.mbicg_params.dummy_rhs.offset, mb.mbicg_params.dummy_seed.offset, mb.mbicg_params.clover.offset,
            mb.mbicg_params.domain_solver.offset, mb.mbicg_params.nssor.offset, mb.mbicg_params.ssor_omega.offset,
            mb.mbicg_stats.host_syncs.offset]
    assert got == want


def test_default_params():
    p = mb.mbicg_default_params()
    assert (p.ncycle, p.nmr, list(p.block)) == (4, 4, [4, 4, 4, 4])
    assert p.mr_mode == mb.MBICG_MR_FROZEN and p.prec_D == mb.MBICG_FP32
    assert p.prec_sap == mb.MBICG_FP32 and p.max_iter == 1000 and p.delta_ru == 0.1
    assert p.clover == 0
    assert (p.domain_solver, p.nssor, p.ssor_omega) == (mb.MBICG_DOMAIN_MR, 1, 1.26)
    q = mb.mbicg_default_params(block=(2, 2, 2, 2), ncycle=1)
    assert list(q.block) == [2, 2, 2, 2] and q.ncycle == 1


def test_create_rejects_bad_dims_without_touching_a_device():
    lib = mb.load_library()
    ctx = ctypes.c_void_p()
    for dims in [(3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 4, -2)]:
        d = (ctypes.c_int * 4)(*dims)
        assert lib.mbicg_create(ctypes.byref(ctx), d, 0, None) == mb.MBICG_EINVAL
        assert not ctx.value
    assert lib.mbicg_create(None, (ctypes.c_int * 4)(4, 4, 4, 4), 0, None) == mb.MBICG_EINVAL
    # NULL contexts are rejected, not dereferenced
    assert lib.mbicg_apply_D(None, None, None, 1, 0.1, 0) == mb.MBICG_EINVAL
    assert lib.mbicg_block_solve(None, None, None, 1, 0.1, 1e-8, None, None, None) == mb.MBICG_EINVAL
    lib.mbicg_destroy(None)


def test_create_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = mb.load_library()
    ctx = ctypes.c_void_p()
    st = lib.mbicg_create(ctypes.byref(ctx), (ctypes.c_int * 4)(4, 4, 4, 4), 0, None)
    assert st == mb.MBICG_ECUDA and not ctx.value


def test_server_rejects_bad_arguments_without_a_device():
    lib = mb.load_library()
    srv = ctypes.c_void_p()
    assert lib.mbicg_server_create(None, 0, 10.0) == mb.MBICG_EINVAL
    assert lib.mbicg_server_create(ctypes.byref(srv), 0, 0.0) == mb.MBICG_EINVAL
    assert lib.mbicg_server_submit(None, 0, None, 1, 0.1, 1e-8, None) == mb.MBICG_EINVAL
    assert lib.mbicg_server_wait(None, 1, None, None, None, None) == mb.MBICG_EINVAL
    assert lib.mbicg_server_stats(None, None, None, None, None) == mb.MBICG_EINVAL
    lib.mbicg_server_destroy(None)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert lib.mbicg_server_create(ctypes.byref(srv), 0, 10.0) == mb.MBICG_ECUDA


def test_a_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: without the CUDA library every call raises instead of
    computing elsewhere."""
    monkeypatch.setattr(mb, "_lib", None)
    monkeypatch.setattr(mb._build, "LIB", str(tmp_path / "libmbicg.so"))
    monkeypatch.setattr(mb._build, "needs_build", lambda: False)
    with pytest.raises(OSError, match="CUDA library not built"):
        mb.load_library()
    with pytest.raises(OSError):
        mb.mbicg_create((4, 4, 4, 4))
    with pytest.raises(OSError):
        mb.mbicg_default_params()


def test_first_loads_from_several_threads_build_once(monkeypatch):
    """Host threads that make their first library call at the same time share
    one load: the build step runs once, and every thread gets the same
    library."""
    import threading
    import time

    real = mb.load_library()
    calls = []

    def build():
        calls.append(1)
        time.sleep(0.2)  # a build takes a while: the other threads arrive meanwhile

    monkeypatch.setattr(mb, "_lib", None)
    monkeypatch.setattr(mb._build, "needs_build", lambda: not calls)
    monkeypatch.setattr(mb._build, "build", build)
    got = [None] * 4
    threads = [threading.Thread(target=lambda i=i: got.__setitem__(i, mb.load_library())) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert len(calls) == 1
    assert all(g is got[0] for g in got) and got[0]._name == real._name
