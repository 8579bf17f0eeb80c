"""The allocation-free operator entry point, mbicg_apply_D_noalloc, for callers
that cannot allocate device memory (stream capture into a CUDA graph, fixed
memory pools).  It must give the result of mbicg_apply_D(..., MBICG_FP32)
within the FP32 operator tolerance of the other tests (1e-6 relative per-site
norm), call after call, although every call reuses the same scratch array.
This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import rel_site_norm

pytestmark = pytest.mark.gpu


def test_noalloc_operator_matches_apply_D_on_consecutive_calls():
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
            assert rel_site_norm(d_out.cpu().numpy(), ref) < 1e-6
    finally:
        mb.mbicg_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    # 16^4 sites with L = 12 need about 170 MiB of scratch, more than the array holds
    with pytest.raises(mb.MbicgError) as e:
        mb.mbicg_apply_D_noalloc((16, 16, 16, 16), small, small, small.clone(), 12, 0.12)
    assert e.value.status == mb.MBICG_EINVAL
    # host pointers are rejected too
    host = np.zeros((8 * 8 * 8 * 16, 4, 3, 1), dtype=np.complex128)
    with pytest.raises(mb.MbicgError):
        mb.mbicg_apply_D_noalloc((8, 8, 8, 16), host, host, host.copy(), 1, 0.12)
