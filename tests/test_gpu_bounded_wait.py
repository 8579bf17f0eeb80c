"""The give-up path of the bounded waits: a wait on bytes that never arrive
returns with its error flag set after its poll limit (about a millisecond
here), the device stays usable, and a wait that completes is not flagged."""
import numpy as np
import pytest

import paper_1104_0737_gb300 as mb
import synth
from gpu_common import make_ctx, rel_site_norm

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_the_context_stays_usable(oracle_mod):
    assert mb.mbicg_selftest_bounded_wait(0, 1 << 12, 16) is True
    assert mb.mbicg_selftest_bounded_wait(0, 1 << 12, 0) is False
    dims, L = (4, 4, 4, 8), 2
    ctx, U = make_ctx(dims, 0.5, seed=71)
    try:
        psi = synth.gaussian_source(dims, L, seed=72)
        out = np.empty_like(psi)
        mb.mbicg_apply_D(ctx, psi, out, L, 0.12, mb.MBICG_FP64)
        assert rel_site_norm(out, oracle_mod.apply_D(dims, U, 0.12, psi)) < 1e-13
    finally:
        mb.mbicg_destroy(ctx)


def test_selftest_rejects_bad_arguments():
    for args in [(0, 0, 16), (0, 1 << 25, 16), (0, 100, 8), (0, 100, -16)]:
        with pytest.raises(mb.MbicgError):
            mb.mbicg_selftest_bounded_wait(*args)
