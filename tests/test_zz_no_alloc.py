"""The allocation-free FP64 sum of phi (lbm_cde_sum_state_noalloc).

It exists for callers that cannot allocate device memory where they need a
conservation check (code running under CUDA graph capture, fixed memory
budgets): its scratch is a static device array instead of a buffer. Here it is
called through the C ABI on states of a running solver and compared with the
solver's own FP64 sum (lbm_cde_sum_phi) on two calls in a row. This file sorts
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from _common import Case, run_gpu
from paper_1404_2363_gb300 import _native as N

pytestmark = pytest.mark.gpu

STORE = {"f32": N.LBM_STORE_F32, "f16": N.LBM_STORE_F16_NEQ, "bf16": N.LBM_STORE_BF16_NEQ}


@pytest.mark.parametrize("lattice,storage", [(9, "f32"), (9, "bf16"), (15, "f32"), (15, "f16")])
def test_noalloc_sum_matches_sum_phi_on_two_calls(lattice, storage):
    L = N.lib()
    if lattice == 9:
        case = Case(storage=storage, nx=300, ny=37, steps=20)
    else:
        case = Case(lattice=15, storage=storage, nx=40, ny=23, nz=17, steps=10,
                    D=np.diag([0.02, 0.03, 0.04]))
    phi0, a, sched = case.inputs()
    _, s = run_gpu(case, phi0, a, sched)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    ncell = int(np.prod(case.shape))
    for _ in range(2):
        s.step(7)
        buf, _t = s.get_state()
        st = L.lbm_cde_sum_state_noalloc(buf.data_ptr(), lattice, STORE[storage], ncell, out.data_ptr(),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == N.LBM_OK, L.lbm_cde_noalloc_last_error()
        torch.cuda.synchronize()
        got = float(out.item())
        ref = s.sum_phi()
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
    s.close()


def test_noalloc_rejects_states_beyond_its_scratch():
    L = N.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    too_big = (1 << 26) + 1   # LBM_NOALLOC_MAX_CELLS + 1
    st = L.lbm_cde_sum_state_noalloc(dummy.data_ptr(), 9, 0, too_big, out.data_ptr(), None)
    assert st == N.LBM_E_ARG
    assert b"exceeds" in L.lbm_cde_noalloc_last_error()
