"""Blocks in page-locked host memory: the library stages them with a copy
kernel that reads the mapped host pages (pageable memory goes through
cudaMemcpyAsync).  Results must be bit for bit those of the same call with
device buffers, for the operator and for a block solve, including a size
that is not a multiple of the copy kernel's four words per thread."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dims,L", [((8, 8, 8, 16), 12), ((4, 4, 4, 6), 1)])
def test_operator_pinned_equals_device(dims, L):
    ctx, U = make_ctx(dims, 0.5, seed=91)
    try:
        x = synth.gaussian_source(dims, L, seed=92)
        hx = torch.from_numpy(x).pin_memory()
        hy = torch.empty_like(hx).pin_memory()
        dx = hx.to("cuda")
        dy = torch.empty_like(dx)
        for prec in (mb.MBICG_FP64, mb.MBICG_FP32):
            mb.mbicg_apply_D(ctx, hx, hy, L, 0.13, prec)
            mb.mbicg_apply_D(ctx, dx, dy, L, 0.13, prec)
            torch.cuda.synchronize()
            assert torch.equal(hy, dy.cpu())
            # pageable numpy memory takes the other path, to the same bits
            y = np.empty_like(x)
            mb.mbicg_apply_D(ctx, x, y, L, 0.13, prec)
            assert np.array_equal(y, hy.numpy())
    finally:
        mb.mbicg_destroy(ctx)


def test_block_solve_pinned_equals_device():
    dims, L = (8, 8, 8, 16), 4
    ctx, U = make_ctx(dims, 0.5, seed=93)
    try:
        B = synth.gaussian_source(dims, L, seed=94)
        p = mb.mbicg_default_params(ncycle=2, nmr=4, block=(4, 4, 4, 4), mr_mode=mb.MBICG_MR_FROZEN)
        hB = torch.from_numpy(B).pin_memory()
        hX = torch.empty_like(hB).pin_memory()
        dB = hB.to("cuda")
        dX = torch.empty_like(dB)
        st1, it1, _ = mb.mbicg_block_solve(ctx, hB, hX, L, 0.125, 1e-10, p)
        st2, it2, _ = mb.mbicg_block_solve(ctx, dB, dX, L, 0.125, 1e-10, p)
        assert st1 == st2 == mb.MBICG_OK and it1 == it2
        assert torch.equal(hX, dX.cpu())
    finally:
        mb.mbicg_destroy(ctx)
