"""The autotuner on the GPU: with MBICG_AUTOTUNE set, the first solve times
the operator's launch configurations (sites per CTA, CTA order) and keeps the
fastest; every configuration computes the same result, so the solve is bit
for bit the one without tuning, and the choice is written to MBICG_TUNE_FILE."""
import os

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def test_tuned_solve_is_bit_identical(tmp_path, monkeypatch):
    dims, L = (8, 8, 8, 16), 4
    ctx, U = make_ctx(dims, 0.5, seed=81)
    try:
        B = synth.gaussian_source(dims, L, seed=82)
        p = mb.mbicg_default_params(ncycle=2, nmr=4, block=(4, 4, 4, 4))
        X0 = np.empty_like(B)
        monkeypatch.delenv("MBICG_AUTOTUNE", raising=False)
        st0, it0, _ = mb.mbicg_block_solve(ctx, B, X0, L, 0.125, 1e-10, p)
        monkeypatch.setenv("MBICG_AUTOTUNE", "1")
        monkeypatch.setenv("MBICG_TUNE_FILE", str(tmp_path / "tune.txt"))
        X1 = np.empty_like(B)
        st1, it1, _ = mb.mbicg_block_solve(ctx, B, X1, L, 0.125, 1e-10, p)
        assert st0 == st1 == mb.MBICG_OK and it0 == it1
        assert np.array_equal(X0, X1)
        lines = (tmp_path / "tune.txt").read_text().split("\n")
        assert any(line.startswith("dslash/fp32/8x8x8x16/L4 ") for line in lines)
        assert any(line.startswith("dslash/fp64/8x8x8x16/L4 ") for line in lines)
    finally:
        mb.mbicg_destroy(ctx)
