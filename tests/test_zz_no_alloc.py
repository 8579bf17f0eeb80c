"""The allocation-free operator entry point, mbicg_apply_D_noalloc, for callers
that cannot allocate device memory (code inside a framework's memory pool,
real-time loops that may not wait for the allocator, programs whose device
memory is fixed at start-up).  It must give the result of
mbicg_apply_D(..., MBICG_FP32), and of the FP64 oracle, within the FP32
operator tolerance of the other tests (1e-6 relative per-site norm), call
after call, although every call reuses the same scratch array.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import rel_site_norm

pytestmark = pytest.mark.gpu


def test_noalloc_operator_matches_apply_D_on_consecutive_calls(oracle_mod):
    torch = pytest.importorskip("torch")
    dims = (8, 8, 8, 16)
    U = synth.su3_links(dims, 0.5, seed=61)
    dU = torch.from_numpy(U).cuda()
    ctx = mb.mbicg_create(dims)
    try:
        mb.mbicg_load_gauge(ctx, U)
        # two calls in a row with different blocks: the second must not see the first's scratch
        for L, kappa, seed in ((12, 0.13, 62), (5, 0.121, 63)):
            psi = synth.gaussian_source(dims, L, seed)
            ref = np.empty_like(psi)
            mb.mbicg_apply_D(ctx, psi, ref, L, kappa, mb.MBICG_FP32)
            d_in = torch.from_numpy(psi).cuda()
            d_out = torch.full_like(d_in, float("nan"))
            mb.mbicg_apply_D_noalloc(dims, dU, d_in, d_out, L, kappa)
            torch.cuda.synchronize()
            got = d_out.cpu().numpy()
            assert rel_site_norm(got, ref) < 1e-6
            assert rel_site_norm(got, oracle_mod.apply_D(dims, U, kappa, psi)) < 1e-6
    finally:
        mb.mbicg_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    dims = (16, 16, 16, 16)
    V = 16 ** 4
    U = torch.zeros(V * 36, dtype=torch.complex128, device="cuda")
    a = torch.zeros(V * 12 * 12, dtype=torch.complex128, device="cuda")
    # 16^4 sites with L = 12 need about 170 MiB of scratch, more than the array holds
    with pytest.raises(mb.MbicgError) as e:
        mb.mbicg_apply_D_noalloc(dims, U, a, a.clone(), 12, 0.12)
    assert e.value.status == mb.MBICG_EINVAL


def test_noalloc_refuses_wrong_buffers_without_launching():
    """Refused on the host, before anything is launched: host memory, buffers
    whose sizes do not match the lattice, in == out."""
    torch = pytest.importorskip("torch")
    dims, L = (8, 8, 8, 16), 2
    V = 8 * 8 * 8 * 16
    U = torch.zeros(V * 36, dtype=torch.complex128, device="cuda")
    a = torch.zeros(V * 12 * L, dtype=torch.complex128, device="cuda")
    host = np.zeros((V, 4, 3, L), dtype=np.complex128)
    with pytest.raises(mb.MbicgError):
        mb.mbicg_apply_D_noalloc(dims, host, host, host.copy(), L, 0.12)
    with pytest.raises(mb.MbicgError):  # U too short
        mb.mbicg_apply_D_noalloc(dims, U[: V * 35], a, a.clone(), L, 0.12)
    with pytest.raises(mb.MbicgError):  # out too short for L columns
        mb.mbicg_apply_D_noalloc(dims, U, a, a[: V * 12].clone(), L, 0.12)
    # the C entry point itself refuses host pointers and aliasing
    lib = mb.load_library()
    import ctypes

    d = (ctypes.c_int * 4)(*dims)
    vp = ctypes.c_void_p
    assert lib.mbicg_apply_D_noalloc(d, vp(host.ctypes.data), vp(a.data_ptr()), vp(a.data_ptr() + 16), L,
                                     0.12, None) == mb.MBICG_EINVAL
    assert lib.mbicg_apply_D_noalloc(d, vp(U.data_ptr()), vp(a.data_ptr()), vp(a.data_ptr()), L,
                                     0.12, None) == mb.MBICG_EINVAL
