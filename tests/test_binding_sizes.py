"""The Python binding refuses, before calling the library, blocks and fields
smaller than the lattice needs: the library reads and writes the full size
through the pointers it is given (device kernels past the end of a device
buffer, host copies past the end of a host array).  No GPU and no library
call: every refusal happens in the binding."""
import ctypes

import numpy as np
import pytest

import paper_1104_0737_gb300 as mb

DIMS = (4, 4, 4, 4)
V = 4 ** 4


def _ctx():
    c = ctypes.c_void_p()
    c.dims = DIMS
    return c


def _block(L, short=0):
    return np.zeros(V * 12 * L - short, dtype=np.complex128)


@pytest.mark.parametrize("call", ["apply_D", "apply_clover", "sap_precond", "block_solve"])
def test_short_blocks_refused(call):
    L = 3
    full, short = _block(L), _block(L, short=1)
    p = mb.mbicg_params()
    fn = {"apply_D": lambda a, b: mb.mbicg_apply_D(_ctx(), a, b, L, 0.12),
          "apply_clover": lambda a, b: mb.mbicg_apply_clover(_ctx(), a, b, L, 0.12),
          "sap_precond": lambda a, b: mb.mbicg_sap_precond(_ctx(), a, b, L, 0.12, p),
          "block_solve": lambda a, b: mb.mbicg_block_solve(_ctx(), a, b, L, 0.12, 1e-10, p)}[call]
    for a, b in ((short, full), (full, short)):
        with pytest.raises(mb.MbicgError) as e:
            fn(a, b)
        assert e.value.status == mb.MBICG_EINVAL


def test_short_field_refused():
    with pytest.raises(mb.MbicgError) as e:
        mb.mbicg_load_gauge(_ctx(), np.zeros(36 * V - 1, dtype=np.complex128))
    assert e.value.status == mb.MBICG_EINVAL
    srv = ctypes.c_void_p()
    srv.field_sites, srv.request_size = {}, {}
    with pytest.raises(mb.MbicgError) as e:
        mb.mbicg_server_add_field(srv, DIMS, np.zeros(36 * V - 1, dtype=np.complex128), mb.mbicg_params())
    assert e.value.status == mb.MBICG_EINVAL


def test_server_blocks_checked_against_the_field_and_request():
    srv = ctypes.c_void_p()
    srv.field_sites, srv.request_size = {0: V}, {5: (12 * V * 2, 2)}
    with pytest.raises(mb.MbicgError) as e:  # B shorter than 2 columns of field 0
        mb.mbicg_server_submit(srv, 0, _block(2, short=1), 2, 0.12, 1e-10)
    assert e.value.status == mb.MBICG_EINVAL
    for X, L in ((_block(2, short=1), 2), (_block(3), 3), (_block(2), 1)):  # short X, or L not the request's
        with pytest.raises(mb.MbicgError) as e:
            mb.mbicg_server_wait(srv, 5, X, L)
        assert e.value.status == mb.MBICG_EINVAL
    assert 5 in srv.request_size  # a refused wait keeps the request


def test_out_of_range_L_left_to_the_library():
    """L outside 1..16 is not size-checked here: the call goes to the library,
    which refuses it (and, here, the stand-in context) itself."""
    a = _block(1)
    with pytest.raises(Exception) as e:
        mb.mbicg_apply_D(_ctx(), a, a.copy(), 17, 0.12)
    assert not (isinstance(e.value, mb.MbicgError) and "lattice needs" in str(e.value))
