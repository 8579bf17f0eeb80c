"""Python binding of libmbicg.so, the GB300 (sm_103a) library for the
modified block BiCGSTAB solve of the Wilson-Dirac equation with SAP
preconditioning (Nakamura et al., arXiv:1104.0737).

The functions carry the names of the C ABI in include/mbicg.h and only
marshal arguments: numpy arrays (host memory) or torch tensors (host or CUDA
memory), complex128 and C-contiguous, in the layouts the header documents.
Every step of the computation runs in the library's CUDA kernels; there is no
other implementation to fall back to, and a missing or unloadable library
raises an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "MBICG_OK", "MBICG_EINVAL", "MBICG_ENOMEM", "MBICG_ENOGAUGE", "MBICG_ENOTCONV",
    "MBICG_EBREAKDOWN", "MBICG_ENAN", "MBICG_ECUDA", "MBICG_FP64", "MBICG_FP32", "MBICG_FP16",
    "MBICG_MR_COLUMN", "MBICG_MR_BLOCK", "MBICG_MR_FROZEN", "MBICG_DOMAIN_MR", "MBICG_DOMAIN_SSOR",
    "KERNEL_CLASSES",
    "MbicgError", "mbicg_params", "mbicg_stats", "library_path", "load_library",
    "mbicg_default_params", "mbicg_create", "mbicg_destroy", "mbicg_load_gauge",
    "mbicg_apply_D", "mbicg_load_clover", "mbicg_apply_clover", "mbicg_sap_precond", "mbicg_sap_table_len",
    "mbicg_sap_precond_frozen", "mbicg_block_solve", "mbicg_get_stats",
    "mbicg_last_error", "mbicg_set_profiling", "mbicg_get_profile", "mbicg_apply_D_noalloc",
    "mbicg_request_info", "mbicg_server_create", "mbicg_server_add_field", "mbicg_server_submit",
    "mbicg_server_wait", "mbicg_server_hold", "mbicg_server_stats", "mbicg_server_memory", "mbicg_server_destroy",
    "mbicg_selftest_bounded_wait",
]

MBICG_OK, MBICG_EINVAL, MBICG_ENOMEM, MBICG_ENOGAUGE = 0, -1, -2, -3
MBICG_ENOTCONV, MBICG_EBREAKDOWN, MBICG_ENAN, MBICG_ECUDA = -4, -5, -6, -7
MBICG_FP64, MBICG_FP32, MBICG_FP16 = 0, 1, 2
MBICG_MR_COLUMN, MBICG_MR_BLOCK, MBICG_MR_FROZEN = 0, 1, 2
MBICG_DOMAIN_MR, MBICG_DOMAIN_SSOR = 0, 1
KERNEL_CLASSES = ["dslash", "dslash64", "sap_resid", "sap_domain", "sap_update", "gram",
                  "axpy", "small", "convert", "sap_sweep"]

_STATUS_NAMES = {0: "MBICG_OK", -1: "MBICG_EINVAL", -2: "MBICG_ENOMEM", -3: "MBICG_ENOGAUGE",
                 -4: "MBICG_ENOTCONV", -5: "MBICG_EBREAKDOWN", -6: "MBICG_ENAN", -7: "MBICG_ECUDA"}


class MbicgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mbicg_params(ctypes.Structure):
    _fields_ = [
        ("ncycle", ctypes.c_int), ("nmr", ctypes.c_int), ("block", ctypes.c_int * 4),
        ("mr_mode", ctypes.c_int), ("prec_sap", ctypes.c_int), ("prec_D", ctypes.c_int),
        ("max_iter", ctypes.c_int), ("use_x0", ctypes.c_int), ("delta_ru", ctypes.c_double),
        ("res_history", ctypes.POINTER(ctypes.c_double)), ("res_history_len", ctypes.c_int),
        ("dummy_rhs", ctypes.c_int), ("dummy_seed", ctypes.c_ulonglong), ("clover", ctypes.c_int),
        ("domain_solver", ctypes.c_int), ("nssor", ctypes.c_int), ("ssor_omega", ctypes.c_double),
    ]


class mbicg_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("restarts", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong), ("true_res_max", ctypes.c_double),
        ("graph_iterations", ctypes.c_int), ("precision_fallbacks", ctypes.c_int), ("host_syncs", ctypes.c_int),
    ]


class mbicg_request_info(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("batch_columns", ctypes.c_int)]


_lib = None
_lib_lock = threading.Lock()  # the first load (and build) happens once, whichever thread asks first


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libmbicg.so (building it first with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is None:
            _lib = _load(build_if_missing)
    return _lib


def _load(build_if_missing: bool):
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise OSError(f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.mbicg_default_params.argtypes = [ctypes.POINTER(mbicg_params)]
    lib.mbicg_default_params.restype = None
    lib.mbicg_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.c_int, vp]
    lib.mbicg_destroy.argtypes = [vp]
    lib.mbicg_destroy.restype = None
    lib.mbicg_load_gauge.argtypes = [vp, vp]
    lib.mbicg_apply_D.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.mbicg_load_clover.argtypes = [vp, ctypes.c_double]
    lib.mbicg_apply_clover.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.mbicg_sap_precond.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(mbicg_params)]
    lib.mbicg_sap_table_len.argtypes = [vp, ctypes.POINTER(mbicg_params), ctypes.POINTER(ctypes.c_longlong)]
    lib.mbicg_sap_precond_frozen.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                             ctypes.POINTER(mbicg_params), dp, ip]
    lib.mbicg_block_solve.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(mbicg_params), ip, dp]
    lib.mbicg_get_stats.argtypes = [vp, ctypes.POINTER(mbicg_stats)]
    lib.mbicg_last_error.argtypes = [vp]
    lib.mbicg_last_error.restype = ctypes.c_char_p
    lib.mbicg_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.mbicg_get_profile.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    lib.mbicg_apply_D_noalloc.argtypes = [ip, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.mbicg_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double]
    lib.mbicg_server_add_field.argtypes = [vp, ip, vp, ctypes.POINTER(mbicg_params), ctypes.c_int, ip]
    lib.mbicg_server_submit.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, llp]
    lib.mbicg_server_wait.argtypes = [vp, ctypes.c_longlong, vp, ip, dp, ctypes.POINTER(mbicg_request_info)]
    lib.mbicg_server_stats.argtypes = [vp, llp, llp, llp, ip]
    lib.mbicg_server_hold.argtypes = [vp, ctypes.c_int]
    lib.mbicg_server_memory.argtypes = [vp, dp, dp, llp]
    lib.mbicg_server_destroy.argtypes = [vp]
    lib.mbicg_server_destroy.restype = None
    lib.mbicg_selftest_bounded_wait.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
    return lib


def _ptr(a, name: str):
    """Data pointer of a C-contiguous complex128 numpy array or torch tensor."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):
        import torch

        if a.dtype != torch.complex128 or not a.is_contiguous():
            raise TypeError(f"{name}: need a contiguous complex128 tensor")
        return ctypes.c_void_p(a.data_ptr()), a.numel()
    import numpy as np

    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError(f"{name}: need a C-contiguous complex128 numpy array or torch tensor")
    return ctypes.c_void_p(a.ctypes.data), a.size


def _need(ctx, name: str, have: int, per_site: int) -> None:
    """Refuses, before the call, a block or field with fewer complex numbers
    than the context's lattice needs (per_site per site): the library reads
    and writes the full size through the pointer, past the end of a shorter
    buffer.  Skipped for a context without recorded extents."""
    dims = getattr(ctx, "dims", None)
    if dims is None:
        return
    V = 1
    for d in dims:
        V *= d
    if have < V * per_site:
        raise MbicgError(MBICG_EINVAL, f"{name}: {have} complex numbers, the lattice needs {V * per_site}")


def _columns_ok(L) -> bool:
    """L within the library's range: only then are block sizes checked here
    (the library itself refuses other L)."""
    return 1 <= int(L) <= 16


def _check(ctx, status: int, allowed=(MBICG_OK,)):
    if status not in allowed:
        raise MbicgError(status, mbicg_last_error(ctx))
    return status


def mbicg_default_params(**overrides) -> mbicg_params:
    p = mbicg_params()
    load_library().mbicg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "block":
            p.block = (ctypes.c_int * 4)(*v)
        else:
            setattr(p, k, v)
    return p


def mbicg_create(dims, device: int = 0, stream=None):
    """Context for a lattice of extents dims = (Lx, Ly, Lz, Lt).  stream: a
    torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    lib = load_library()
    ctx = ctypes.c_void_p()
    raw = None
    if stream is not None:
        raw = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    st = lib.mbicg_create(ctypes.byref(ctx), d, int(device), raw)
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_create failed")
    ctx.dims = tuple(int(x) for x in dims)
    return ctx


def mbicg_destroy(ctx) -> None:
    load_library().mbicg_destroy(ctx)


def mbicg_last_error(ctx) -> str:
    return load_library().mbicg_last_error(ctx).decode()


def mbicg_load_gauge(ctx, U) -> None:
    p, n = _ptr(U, "U")
    _need(ctx, "U", n, 36)
    _check(ctx, load_library().mbicg_load_gauge(ctx, p))


def mbicg_apply_D(ctx, inp, out, L: int, kappa: float, prec: int = MBICG_FP64) -> None:
    pi, ni = _ptr(inp, "in")
    po, no = _ptr(out, "out")
    if _columns_ok(L):
        _need(ctx, "in", ni, 12 * int(L))
        _need(ctx, "out", no, 12 * int(L))
    _check(ctx, load_library().mbicg_apply_D(ctx, pi, po, int(L), float(kappa), int(prec)))


def mbicg_load_clover(ctx, csw: float) -> None:
    _check(ctx, load_library().mbicg_load_clover(ctx, float(csw)))


def mbicg_apply_clover(ctx, inp, out, L: int, kappa: float, prec: int = MBICG_FP64, jacobi: int = 0) -> None:
    pi, ni = _ptr(inp, "in")
    po, no = _ptr(out, "out")
    if _columns_ok(L):
        _need(ctx, "in", ni, 12 * int(L))
        _need(ctx, "out", no, 12 * int(L))
    _check(ctx, load_library().mbicg_apply_clover(ctx, pi, po, int(L), float(kappa), int(prec), int(jacobi)))


def mbicg_sap_precond(ctx, inp, out, L: int, kappa: float, params: mbicg_params) -> None:
    pi, ni = _ptr(inp, "in")
    po, no = _ptr(out, "out")
    if _columns_ok(L):
        _need(ctx, "in", ni, 12 * int(L))
        _need(ctx, "out", no, 12 * int(L))
    _check(ctx, load_library().mbicg_sap_precond(ctx, pi, po, int(L), float(kappa),
                                                 ctypes.byref(params)))


def mbicg_sap_table_len(ctx, params: mbicg_params) -> int:
    """Doubles in the step-length table of mbicg_sap_precond_frozen."""
    n = ctypes.c_longlong(0)
    _check(ctx, load_library().mbicg_sap_table_len(ctx, ctypes.byref(params), ctypes.byref(n)))
    return n.value


def mbicg_sap_precond_frozen(ctx, inp, out, L: int, kappa: float, params: mbicg_params, table) -> bool:
    """out = M_SAP in with frozen step lengths held in `table` (host numpy
    complex128, ncycle * 2 * nmr * n_domains entries, NaN = not yet recorded;
    recorded entries are written back).  Returns True when every entry the
    sweeps use is set."""
    import numpy as np

    pi, ni = _ptr(inp, "in")
    po, no = _ptr(out, "out")
    if _columns_ok(L):
        _need(ctx, "in", ni, 12 * int(L))
        _need(ctx, "out", no, 12 * int(L))
    n = mbicg_sap_table_len(ctx, params)
    if (not isinstance(table, np.ndarray) or table.dtype != np.complex128 or not table.flags.c_contiguous
            or 2 * table.size != n):
        raise TypeError(f"table: need a C-contiguous complex128 numpy array of {n // 2} entries")
    done = ctypes.c_int(0)
    _check(ctx, load_library().mbicg_sap_precond_frozen(
        ctx, pi, po, int(L), float(kappa), ctypes.byref(params),
        table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(done)))
    return bool(done.value)


def mbicg_block_solve(ctx, B, X, L: int, kappa: float, tol: float, params: mbicg_params):
    """Returns (status, iters, true_res list).  MBICG_ENOTCONV and
    MBICG_EBREAKDOWN are returned (X and true_res are filled); every other
    failure raises MbicgError."""
    pb, nb = _ptr(B, "B")
    px, nx = _ptr(X, "X")
    if _columns_ok(L):
        _need(ctx, "B", nb, 12 * int(L))
        _need(ctx, "X", nx, 12 * int(L))
    iters = ctypes.c_int(0)
    tres = (ctypes.c_double * max(1, int(L)))()
    st = load_library().mbicg_block_solve(ctx, pb, px, int(L), float(kappa), float(tol),
                                          ctypes.byref(params), ctypes.byref(iters), tres)
    _check(ctx, st, (MBICG_OK, MBICG_ENOTCONV, MBICG_EBREAKDOWN))
    return st, iters.value, [tres[i] for i in range(int(L))]


def mbicg_get_stats(ctx) -> dict:
    s = mbicg_stats()
    _check(ctx, load_library().mbicg_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in mbicg_stats._fields_}


def mbicg_set_profiling(ctx, enable: bool) -> None:
    _check(ctx, load_library().mbicg_set_profiling(ctx, int(bool(enable))))


def mbicg_get_profile(ctx) -> dict:
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(ctx, load_library().mbicg_get_profile(ctx, ms, cnt, n))
    return {KERNEL_CLASSES[i]: (ms[i], cnt[i]) for i in range(n)}


def mbicg_apply_D_noalloc(dims, U, inp, out, L: int, kappa: float, stream=None) -> None:
    """out = A in (FP32) without any allocation, for callers that cannot
    allocate device memory (inside a framework's memory pool, real-time loops
    that may not wait for the allocator, device memory fixed at start-up).
    U, inp, out: CUDA tensors on the current device with V*36 and V*12*L
    elements.  Ordered on `stream` (torch.cuda.Stream, raw handle or None);
    returns without waiting.  Concurrent calls share one scratch array and race."""
    V = 1
    for d in dims:
        V *= int(d)
    pu, nu = _ptr(U, "U")
    pi, ni = _ptr(inp, "in")
    po, no = _ptr(out, "out")
    if nu != V * 36 or ni != V * 12 * int(L) or no != V * 12 * int(L):
        raise MbicgError(MBICG_EINVAL, f"mbicg_apply_D_noalloc: U needs {V * 36} and in/out {V * 12 * int(L)} "
                                       f"complex numbers, got {nu}, {ni}, {no}")
    for t, name in ((U, "U"), (inp, "in"), (out, "out")):
        if not getattr(t, "is_cuda", False):
            raise MbicgError(MBICG_EINVAL, f"mbicg_apply_D_noalloc: {name} must be a CUDA tensor")
        import torch

        if t.device.index != torch.cuda.current_device():
            raise MbicgError(MBICG_EINVAL, f"mbicg_apply_D_noalloc: {name} is not on the current device")
    raw = None
    if stream is not None:
        raw = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    st = load_library().mbicg_apply_D_noalloc(d, pu, pi, po, int(L), float(kappa), raw)
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_apply_D_noalloc failed (sizes beyond the scratch, pointers not on the "
                             "current device, or a CUDA error)")


def _host(a, name: str):
    import numpy as np

    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError(f"{name}: need a C-contiguous complex128 numpy array (host memory)")
    return ctypes.c_void_p(a.ctypes.data)


def mbicg_server_create(device: int = 0, hbm_budget_gb: float = 100.0):
    """A request server on `device` whose solver slots may take hbm_budget_gb
    gigabytes of device memory."""
    srv = ctypes.c_void_p()
    st = load_library().mbicg_server_create(ctypes.byref(srv), int(device), float(hbm_budget_gb))
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_server_create failed")
    # sites per field and complex numbers per request, for the size checks of
    # submit and wait (the library copies the full block through the pointer)
    srv.field_sites = {}
    srv.request_size = {}
    return srv


def mbicg_server_add_field(server, dims, U, params: mbicg_params, max_slots: int = 1) -> int:
    """Makes the gauge field U (host numpy) resident with up to max_slots
    solver slots; returns its field id."""
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    V = 1
    for x in dims:
        V *= int(x)
    pu = _host(U, "U")
    if U.size < 36 * V:
        raise MbicgError(MBICG_EINVAL, f"mbicg_server_add_field: U has {U.size} complex numbers, "
                                       f"the lattice needs {36 * V}")
    fid = ctypes.c_int(-1)
    st = load_library().mbicg_server_add_field(server, d, pu, ctypes.byref(params),
                                               int(max_slots), ctypes.byref(fid))
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_server_add_field failed (HBM budget, bad dims or a CUDA error)")
    if hasattr(server, "field_sites"):
        server.field_sites[fid.value] = V
    return fid.value


def mbicg_server_submit(server, field: int, B, L: int, kappa: float, tol: float) -> int:
    """Queues A X = B (host numpy, L columns, copied now); returns the request id."""
    rid = ctypes.c_longlong(0)
    pb = _host(B, "B")
    V = getattr(server, "field_sites", {}).get(int(field))
    if V is not None and 1 <= int(L) <= 12 and B.size < 12 * V * int(L):
        raise MbicgError(MBICG_EINVAL, f"mbicg_server_submit: B has {B.size} complex numbers, "
                                       f"{L} columns need {12 * V * int(L)}")
    st = load_library().mbicg_server_submit(server, int(field), pb, int(L), float(kappa),
                                            float(tol), ctypes.byref(rid))
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_server_submit: unknown field, L outside 1..12, tol <= 0, or a block "
                             "that can never fit in the memory budget")
    if V is not None:
        server.request_size[rid.value] = (12 * V * int(L), int(L))
    return rid.value


def mbicg_server_wait(server, request_id: int, X, L: int):
    """Blocks until the request is solved; fills X (host numpy, its L columns).
    Returns (status, iters, true_res list, info dict)."""
    it = ctypes.c_int(0)
    tres = (ctypes.c_double * max(1, int(L)))()
    info = mbicg_request_info()
    px = _host(X, "X")
    known = getattr(server, "request_size", {}).get(int(request_id))
    if known is not None and (X.size < known[0] or int(L) != known[1]):
        raise MbicgError(MBICG_EINVAL, f"mbicg_server_wait: the request has {known[1]} columns "
                                       f"({known[0]} complex numbers); got L = {L} and X of {X.size}")
    st = load_library().mbicg_server_wait(server, int(request_id), px, ctypes.byref(it), tres,
                                          ctypes.byref(info))
    if known is not None and st != MBICG_EINVAL:
        server.request_size.pop(int(request_id), None)
    if st not in (MBICG_OK, MBICG_ENOTCONV, MBICG_EBREAKDOWN):
        raise MbicgError(st, "mbicg_server_wait: unknown request or a failed block solve")
    return st, it.value, [tres[i] for i in range(int(L))], {k: getattr(info, k) for k, _ in info._fields_}


def mbicg_server_hold(server, hold: bool) -> None:
    """While held, no slot starts a new block solve; releasing lets the slots
    pack everything that waits."""
    st = load_library().mbicg_server_hold(server, int(bool(hold)))
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_server_hold failed")


def mbicg_server_stats(server) -> dict:
    a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    n = ctypes.c_int()
    load_library().mbicg_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n))
    return {"solves": a.value, "columns": b.value, "max_columns": c.value, "slots": n.value}


def mbicg_server_memory(server) -> dict:
    """Device memory held (GB), the budget (GB) and the waits for memory."""
    u, b, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    load_library().mbicg_server_memory(server, ctypes.byref(u), ctypes.byref(b), ctypes.byref(w))
    return {"used_gb": u.value, "budget_gb": b.value, "memory_waits": w.value}


def mbicg_server_destroy(server) -> None:
    load_library().mbicg_server_destroy(server)


def mbicg_selftest_bounded_wait(device: int = 0, spin_limit: int = 1 << 12, expect_bytes: int = 16) -> bool:
    """Runs the kernels' bounded mbarrier wait on a barrier whose bytes never
    arrive (expect_bytes > 0) or that completes (0); True when it gave up."""
    out = ctypes.c_int(-1)
    st = load_library().mbicg_selftest_bounded_wait(int(device), int(spin_limit), int(expect_bytes),
                                                    ctypes.byref(out))
    if st != MBICG_OK:
        raise MbicgError(st, "mbicg_selftest_bounded_wait failed")
    return bool(out.value)
