"""Shared set-up of the GPU parity tests: seeded inputs from synth, a context
with the gauge field loaded through the C ABI."""
import numpy as np

import paper_1104_0737_gb300 as mb
import synth


def make_ctx(dims, eps=0.5, seed=1000):
    U = synth.su3_links(dims, eps, seed)
    ctx = mb.mbicg_create(dims)
    mb.mbicg_load_gauge(ctx, U)
    return ctx, U


def rel_site_norm(a, b):
    """max over sites of |a_x - b_x| / |b_x| (norm over spin, colour and rhs)."""
    V = a.shape[0]
    d = np.linalg.norm((a - b).reshape(V, -1), axis=1)
    r = np.linalg.norm(b.reshape(V, -1), axis=1)
    return float(np.max(d / r))


def rel_col_norm(a, b):
    """max over columns of |a_i - b_i| / |b_i|."""
    L = a.shape[-1]
    d = np.linalg.norm((a - b).reshape(-1, L), axis=0)
    r = np.linalg.norm(b.reshape(-1, L), axis=0)
    return float(np.max(d / r))
