"""Parity of the solver's own preconditioner with the FP64 oracle: SAP with
frozen MR step lengths (Sec. 2.1 asks for a stationary M; Sec. 2.2 defines
M_SAP), through mbicg_sap_precond_frozen.

Each case runs the sequence a block solve goes through: a point source first
(only the domains its residual reaches record their step lengths), then a
Gaussian source (the rest of the table fills), then replays of the complete
table by the fused on-chip sweep.  The oracle runs the same sequence with its
own table.  The replay kernel is also given the oracle's own table, so that
both sides apply exactly the same linear operator M; outputs are compared
site by site (1e-5 in FP32, 1e-12 in FP64), and the recorded tables entry by
entry."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def site_err(out, ref):
    """max over sites of |out_x - ref_x| / |ref_x| where ref_x != 0; sites
    where the oracle's result is exactly zero must be exactly zero."""
    V = ref.shape[0]
    r = np.linalg.norm(ref.reshape(V, -1), axis=1)
    d = np.linalg.norm((out - ref).reshape(V, -1), axis=1)
    nz = r > 0
    assert np.all(d[~nz] == 0), "nonzero result where the oracle's is zero"
    return float(np.max(d[nz] / r[nz])) if nz.any() else 0.0


def table_err(tg, to):
    """The same entries recorded (NaN pattern) and their relative difference."""
    assert np.array_equal(np.isnan(tg), np.isnan(to)), "different entries recorded"
    m = ~np.isnan(to)
    return float(np.max(np.abs(tg[m] - to[m]) / np.maximum(np.abs(to[m]), 1e-300))) if m.any() else 0.0


def domain_colours(dims, block):
    """Checkerboard colour of every domain, numbered lexicographically."""
    nb = [d // b for d, b in zip(dims, block)]
    i = np.arange(int(np.prod(nb)))
    b0 = i % nb[0]
    b1 = (i // nb[0]) % nb[1]
    b2 = (i // (nb[0] * nb[1])) % nb[2]
    b3 = i // (nb[0] * nb[1] * nb[2])
    return (b0 + b1 + b2 + b3) & 1


def run_sequence(oracle_mod, dims, block, L, ncycle, nmr, kappa, prec, tol, seed):
    ctx, U = make_ctx(dims, 0.5, seed=seed)
    try:
        p = mb.mbicg_default_params(ncycle=ncycle, nmr=nmr, block=block, mr_mode=mb.MBICG_MR_FROZEN,
                                    prec_sap=prec)
        nd = int(np.prod(dims)) // int(np.prod(block))
        assert mb.mbicg_sap_table_len(ctx, p) == 2 * ncycle * 2 * nmr * nd
        tg = np.full((ncycle, 2, nmr, nd), np.nan, dtype=np.complex128)
        to = tg.copy()
        colour_of = domain_colours(dims, block)

        def complete(t):
            return all(not np.isnan(t[:, c, :, colour_of == c]).any() for c in (0, 1))
        point = synth.point_source(dims, L)
        gauss = synth.gaussian_source(dims, L, seed=seed + 1)
        gauss2 = synth.gaussian_source(dims, L, seed=seed + 2)
        out = np.empty_like(gauss)

        # 1. point source: a partial table
        done = mb.mbicg_sap_precond_frozen(ctx, point, out, L, kappa, p, tg)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, point, mr_mode=2, omega_table=to)
        assert site_err(out, ref) < tol
        assert table_err(tg, to) < tol
        assert done == complete(to)
        # 2. Gaussian source: the rest of the table
        done = mb.mbicg_sap_precond_frozen(ctx, gauss, out, L, kappa, p, tg)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, gauss, mr_mode=2, omega_table=to)
        assert done
        assert site_err(out, ref) < tol
        assert table_err(tg, to) < tol
        # the entries of the other colour stay unused
        for c in (0, 1):
            assert np.isnan(tg[:, c, :, colour_of != c]).all()
            assert not np.isnan(tg[:, c, :, colour_of == c]).any()
        # 3. replay of the library's table, a new source
        done = mb.mbicg_sap_precond_frozen(ctx, gauss2, out, L, kappa, p, tg)
        ref = oracle_mod.sap(dims, block, U, kappa, ncycle, nmr, gauss2, mr_mode=2, omega_table=to)
        assert done
        assert site_err(out, ref) < tol
        # 4. replay of the oracle's own table: the same linear operator on both sides
        tx = to.copy()
        mb.mbicg_sap_precond_frozen(ctx, gauss2, out, L, kappa, p, tx)
        assert np.array_equal(tx, to, equal_nan=True)  # a complete table is not touched
        assert site_err(out, ref) < tol
        # 5. linearity of the replayed M (the stationary preconditioner of Sec. 2.1)
        out2 = np.empty_like(out)
        mb.mbicg_sap_precond_frozen(ctx, np.ascontiguousarray(2.5 * gauss2), out2, L, kappa, p, tx)
        assert site_err(out2, 2.5 * ref) < tol
    finally:
        mb.mbicg_destroy(ctx)


CASES = [
    # dims, block, L, ncycle, nmr, kappa: 8^4 domains (the benchmark's, 8-CTA cluster sweep)
    ((16, 16, 16, 16), (8, 8, 8, 8), 12, 2, 4, 0.146),
    # 4^4 domains (the one-CTA sweep) on 8^3 x 16; two cycles keep the point
    # source's far values, and their MR sums, inside FP32's normal range
    ((8, 8, 8, 16), (4, 4, 4, 4), 12, 2, 4, 0.125),
    # a domain shape the fused sweep does not take: multi-kernel replay
    ((8, 8, 8, 8), (2, 4, 2, 4), 3, 2, 3, 0.13),
]


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,kappa", CASES)
def test_frozen_sap_fp32_matches_oracle(oracle_mod, monkeypatch, dims, block, L, ncycle, nmr, kappa):
    monkeypatch.setenv("MBICG_SAP_FUSED", "1")
    run_sequence(oracle_mod, dims, block, L, ncycle, nmr, kappa, mb.MBICG_FP32, 1e-5, 41)


@pytest.mark.parametrize("dims,block,L,ncycle,nmr,kappa", [((8, 8, 8, 16), (4, 4, 4, 4), 4, 2, 4, 0.125)])
def test_frozen_sap_fp64_matches_oracle(oracle_mod, dims, block, L, ncycle, nmr, kappa):
    run_sequence(oracle_mod, dims, block, L, ncycle, nmr, kappa, mb.MBICG_FP64, 1e-12, 43)


def test_frozen_sap_rejects_bad_tables():
    dims = (8, 8, 8, 8)
    ctx, _ = make_ctx(dims, 0.5, seed=5)
    try:
        eta = synth.gaussian_source(dims, 2, seed=6)
        out = np.empty_like(eta)
        p = mb.mbicg_default_params(ncycle=1, nmr=2, block=(4, 4, 4, 4), mr_mode=mb.MBICG_MR_FROZEN)
        with pytest.raises(TypeError):  # wrong length
            mb.mbicg_sap_precond_frozen(ctx, eta, out, 2, 0.12, p, np.zeros(3, dtype=np.complex128))
        p2 = mb.mbicg_default_params(ncycle=1, nmr=2, block=(4, 4, 4, 4), mr_mode=mb.MBICG_MR_BLOCK)
        t = np.full(mb.mbicg_sap_table_len(ctx, p2) // 2, np.nan, dtype=np.complex128)
        with pytest.raises(mb.MbicgError) as e:  # a table needs the frozen mode
            mb.mbicg_sap_precond_frozen(ctx, eta, out, 2, 0.12, p2, t)
        assert e.value.status == mb.MBICG_EINVAL
    finally:
        mb.mbicg_destroy(ctx)


@pytest.mark.slow
def test_frozen_sap_full_size_32c64_L12(oracle_mod, monkeypatch):
    """The benchmark's lattice and launch configuration (32^3 x 64, 8^4
    domains on 8-CTA clusters, L = 12, FP32): a point source, then a Gaussian
    source recording the rest of the table, then the replay of the oracle's
    table by the fused sweep; one cycle of three MR steps keeps the oracle
    within a few minutes."""
    monkeypatch.setenv("MBICG_SAP_FUSED", "1")
    dims, block, L, kappa = (32, 32, 32, 64), (8, 8, 8, 8), 12, 0.14774
    ctx, U = make_ctx(dims, 0.5, seed=1003)
    try:
        p = mb.mbicg_default_params(ncycle=1, nmr=3, block=block, mr_mode=mb.MBICG_MR_FROZEN,
                                    prec_sap=mb.MBICG_FP32)
        nd = int(np.prod(dims)) // int(np.prod(block))
        tg = np.full((1, 2, 3, nd), np.nan, dtype=np.complex128)
        to = tg.copy()
        point = synth.point_source(dims, L)
        out = np.empty_like(point)
        mb.mbicg_sap_precond_frozen(ctx, point, out, L, kappa, p, tg)
        ref = oracle_mod.sap(dims, block, U, kappa, 1, 3, point, mr_mode=2, omega_table=to)
        assert site_err(out, ref) < 1e-5
        assert table_err(tg, to) < 1e-5
        del point
        gauss = synth.gaussian_source(dims, L, seed=2003)
        assert mb.mbicg_sap_precond_frozen(ctx, gauss, out, L, kappa, p, tg)
        ref = oracle_mod.sap(dims, block, U, kappa, 1, 3, gauss, mr_mode=2, omega_table=to)
        assert site_err(out, ref) < 1e-5
        assert table_err(tg, to) < 1e-5
        # the oracle's table replayed by the fused sweep
        tx = to.copy()
        mb.mbicg_sap_precond_frozen(ctx, gauss, out, L, kappa, p, tx)
        assert site_err(out, ref) < 1e-5
    finally:
        mb.mbicg_destroy(ctx)
