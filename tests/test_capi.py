"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/lbm_cde.h declares, and rejects bad descriptors before any
device work."""
import ctypes

import pytest

from paper_1404_2363_gb300 import _native as N


@pytest.fixture(scope="module")
def L():
    return N.lib()


def test_every_declared_symbol_is_exported(L):
    names = N.header_symbols()
    assert "lbm_cde_step" in names and "lbm_cde_set_D" in names
    for n in names:
        assert hasattr(L, n), n


def test_desc_init_defaults(L):
    d = N.LbmDesc()
    assert L.lbm_cde_desc_init(ctypes.byref(d), 9, 64, 32, 1) == N.LBM_OK
    assert (d.lattice, d.nx, d.ny, d.nz) == (9, 64, 32, 1)
    assert d.storage == N.LBM_STORE_F32 and d.tie_q_rates == 1
    assert d.alpha1 != d.alpha1  # NaN selects the defaults


@pytest.mark.parametrize("field,value", [("lattice", 7), ("nz", 2), ("storage", 5), ("bc_lo_y", 9), ("ny", 0)])
def test_bad_descriptors_rejected_before_device_work(L, field, value):
    d = N.LbmDesc()
    L.lbm_cde_desc_init(ctypes.byref(d), 9, 64, 32, 1)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert L.lbm_cde_create(ctypes.byref(d), ctypes.byref(h)) == N.LBM_E_ARG
    assert h.value is None
    assert len(L.lbm_cde_last_error(None)) > 0


def test_mixed_periodic_walls_rejected(L):
    d = N.LbmDesc()
    L.lbm_cde_desc_init(ctypes.byref(d), 9, 64, 32, 1)
    d.bc_lo_y = N.LBM_BC_NOFLUX_NODE
    h = ctypes.c_void_p()
    assert L.lbm_cde_create(ctypes.byref(d), ctypes.byref(h)) == N.LBM_E_ARG


def test_null_handle_calls(L):
    assert L.lbm_cde_step(None, 1) == N.LBM_E_ARG
    assert L.lbm_cde_destroy(None) == N.LBM_OK
    assert L.lbm_cde_set_wait_limit(None, 100) == N.LBM_E_ARG
    assert L.lbm_cde_set_launch(None, 128, 7) == N.LBM_E_ARG
    assert L.lbm_cde_sync(None) == N.LBM_E_ARG
