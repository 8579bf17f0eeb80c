"""The fused SAP sweep's launch shapes on 8^4 domains (clusters of 8 CTAs with
one column per thread, of 16 CTAs with two columns or one), forced one at a
time with MBICG_SWEEP_SHAPE.  Every shape sums each column's hops in the same
order, so with frozen step lengths (Sec. 2.1's stationary M, the solver's
mode) they agree bit for bit: the replay of the oracle's table, FP32 and FP16
storage, an even and an odd number of columns (the two-column shape's last
group then holds one), and whole block solves.  The autotuner records its
choice of shape under a "sap_sweep/" key."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

SHAPES = (0, 1, 2)


def site_err(out, ref):
    V = ref.shape[0]
    r = np.linalg.norm(ref.reshape(V, -1), axis=1)
    d = np.linalg.norm((out - ref).reshape(V, -1), axis=1)
    return float(np.max(d / r))


@pytest.mark.parametrize("L", [12, 5])
@pytest.mark.parametrize("prec", [mb.MBICG_FP32, mb.MBICG_FP16])
def test_shapes_replay_the_oracles_table_bit_identically(oracle_mod, monkeypatch, L, prec):
    monkeypatch.setenv("MBICG_SAP_FUSED", "1")
    dims, block, ncycle, nmr, kappa = (16, 16, 16, 16), (8, 8, 8, 8), 2, 4, 0.146
    ctx, U = make_ctx(dims, 0.5, seed=61)
    try:
        nd = int(np.prod(dims)) // int(np.prod(block))
        to = np.full((ncycle, 2, nmr, nd), np.nan, dtype=np.complex128)
        oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, synth.gaussian_source(dims, L, seed=62), mr_mode=2,
                       omega_table=to)
        eta = synth.gaussian_source(dims, L, seed=63)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, eta, mr_mode=2, omega_table=to)
        p = mb.mbicg_default_params(ncycle=ncycle, nmr=nmr, block=block, mr_mode=mb.MBICG_MR_FROZEN, prec_sap=prec)
        outs = []
        for shape in SHAPES:
            monkeypatch.setenv("MBICG_SWEEP_SHAPE", str(shape))
            out = np.empty_like(eta)
            assert mb.mbicg_sap_precond_frozen(ctx, eta, out, L, kappa, p, to.copy())
            outs.append(out)
        for out in outs[1:]:
            assert np.array_equal(out, outs[0])
        # FP16 storage: (2 + 4 ncycle) roundings of 2^-11 (test_gpu_sap_fp16)
        assert site_err(outs[0], ref) < (1e-5 if prec == mb.MBICG_FP32 else 2e-2)
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.slow
def test_shapes_give_the_same_block_solve(monkeypatch):
    """16^3 x 32, L = 12 Gaussian sources, kappa 0.128, the benchmark's SAP
    (8^4 domains, 4 cycles, 4 MR steps, frozen): the same iterations and the
    same X, bit for bit, whatever the sweep's shape."""
    dims, L, kappa = (16, 16, 16, 32), 12, 0.128
    ctx, U = make_ctx(dims, 0.5, seed=1002)
    try:
        B = synth.gaussian_source(dims, L, seed=2002)
        p = mb.mbicg_default_params(ncycle=4, nmr=4, block=(8, 8, 8, 8), mr_mode=mb.MBICG_MR_FROZEN,
                                    prec_D=mb.MBICG_FP32, max_iter=2000)
        res = []
        for shape in SHAPES:
            monkeypatch.setenv("MBICG_SWEEP_SHAPE", str(shape))
            X = np.empty_like(B)
            st, it, tres = mb.mbicg_block_solve(ctx, B, X, L, kappa, 1e-10, p)
            assert st == mb.MBICG_OK and max(tres) <= 1e-10
            res.append((it, X))
        for it, X in res[1:]:
            assert it == res[0][0]
            assert np.array_equal(X, res[0][1])
    finally:
        mb.mbicg_destroy(ctx)


def test_autotuner_records_the_sweep_shape(tmp_path, monkeypatch):
    dims, L = (16, 16, 16, 16), 4
    ctx, U = make_ctx(dims, 0.5, seed=64)
    try:
        B = synth.gaussian_source(dims, L, seed=65)
        p = mb.mbicg_default_params(ncycle=2, nmr=4, block=(8, 8, 8, 8), mr_mode=mb.MBICG_MR_FROZEN)
        monkeypatch.delenv("MBICG_SWEEP_SHAPE", raising=False)
        monkeypatch.delenv("MBICG_AUTOTUNE", raising=False)
        X0 = np.empty_like(B)
        st0, it0, _ = mb.mbicg_block_solve(ctx, B, X0, L, 0.13, 1e-10, p)
        monkeypatch.setenv("MBICG_AUTOTUNE", "1")
        monkeypatch.setenv("MBICG_TUNE_FILE", str(tmp_path / "tune.txt"))
        X1 = np.empty_like(B)
        st1, it1, _ = mb.mbicg_block_solve(ctx, B, X1, L, 0.13, 1e-10, p)
        assert st0 == st1 == mb.MBICG_OK and it0 == it1
        assert np.array_equal(X0, X1)
        lines = (tmp_path / "tune.txt").read_text().split("\n")
        hit = [line for line in lines if line.startswith("sap_sweep/fp32/16x16x16x16/L4 ")]
        assert len(hit) == 1 and int(hit[0].split()[1]) in SHAPES
    finally:
        mb.mbicg_destroy(ctx)
