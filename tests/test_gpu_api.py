"""GPU checks of the C-ABI behaviour: determinism, checkpoint/resume,
conservation, the host round trip, error statuses."""
import numpy as np
import pytest
import torch

from _common import Case, rel_l2, run_gpu
from paper_1404_2363_gb300 import _native as N
from paper_1404_2363_gb300.solver import Solver

pytestmark = pytest.mark.gpu


def test_bitwise_deterministic():
    case = Case()
    phi0, a, sched = case.inputs()
    r1, _ = run_gpu(case, phi0, a, sched)
    r2, _ = run_gpu(case, phi0, a, sched)
    assert np.array_equal(r1, r2)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_checkpoint_resume_is_bit_exact(storage):
    case = Case(storage=storage)
    phi0, a, sched = case.inputs()
    ref, _ = run_gpu(case, phi0, a, sched, steps=120)
    _, s = run_gpu(case, phi0, a, sched, steps=50)
    buf, t = s.get_state()
    host = buf.cpu()
    s.step(30)                      # diverge, then restore
    s.set_state(host.cuda(), t)
    assert s.t == 50
    s.step(70)
    assert np.array_equal(s.get_phi().cpu().numpy().astype(np.float64), ref)


def test_conservation_periodic_fp64_sum():
    case = Case(nx=512, ny=256, steps=400)
    phi0, a, sched = case.inputs()
    _, s = run_gpu(case, phi0, a, sched)
    m0 = float(phi0.astype(np.float64).sum())
    assert abs(s.sum_phi() - m0) / m0 < 2e-6


def test_run_host_matches_device_path():
    case = Case(steps=80)
    phi0, a, sched = case.inputs()
    ref, s = run_gpu(case, phi0, a, sched)
    out = s.run_host(phi0, case.steps)
    assert np.array_equal(out.astype(np.float64), ref)


def test_not_spd_rejected():
    s = Solver(nx=64, ny=32)
    with pytest.raises(N.LbmError) as e:
        s.set_D(np.array([[0.02, 0.03], [0.03, 0.02]]))
    assert e.value.status == N.LBM_E_NOT_SPD
    with pytest.raises(N.LbmError) as e:
        s.set_D(np.array([[0.02, 0.01], [0.0, 0.02]]))
    assert e.value.status == N.LBM_E_NOT_SPD


def test_step_before_set_phi_is_state_error():
    s = Solver(nx=64, ny=32)
    s.set_D(np.eye(2) * 0.02)
    with pytest.raises(N.LbmError) as e:
        s.step(1)
    assert e.value.status == N.LBM_E_STATE


def test_nonfinite_phi_reported():
    """A NaN injected in phi0 on the host surfaces as LBM_E_NONFINITE."""
    s = Solver(nx=64, ny=32)
    s.set_D(np.eye(2) * 0.02)
    phi = torch.ones(32, 64, device="cuda")
    phi[5, 7] = float("nan")
    s.set_phi(phi)
    s.step(3)
    with pytest.raises(N.LbmError) as e:
        s.sum_phi()
    assert e.value.status == N.LBM_E_NONFINITE


def test_rates_follow_eq36():
    import oracle as O

    s = Solver(nx=16, ny=16)
    D = np.array([[0.02, 0.01], [0.01, 0.04]])
    s.set_D(D)
    A, rates = s.rates()
    assert np.allclose(A, O.A_from_D(D), rtol=1e-12)
    assert abs(rates[4] - A[0, 0]) < 1e-6 and abs(rates[6] - A[1, 1]) < 1e-6


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_zero_steps_are_a_no_op_and_negative_counts_rejected(storage):
    case = Case(storage=storage, steps=7)
    phi0, a, sched = case.inputs()
    got, s = run_gpu(case, phi0, a, sched)
    s.step(0)
    assert np.array_equal(s.get_phi().cpu().numpy(), got)
    with pytest.raises(N.LbmError) as e:
        s.step(-1)
    assert e.value.status == N.LBM_E_ARG
    s.step(1)                      # the handle is still usable
    assert np.isfinite(s.get_phi().cpu().numpy()).all()
    s.close()


def test_batch_zero_steps_are_a_no_op_and_negative_counts_rejected():
    from paper_1404_2363_gb300.batch import Batch, poiseuille_row

    u = poiseuille_row(9, 0.05)
    ch = {"nx": 64, "ny": 9, "bc": ("noflux", "noflux"), "D": [[0.02, 0.0], [0.0, 0.02]], "u_row": u,
          "x_ref0": 20.0, "x_ref_velocity": 0.0}
    phi = np.random.default_rng(2).uniform(0.5, 1.5, (9, 64)).astype(np.float32)
    b = Batch([ch, dict(ch, nx=96)], graph_steps=4)
    b.set_phi([phi, np.tile(phi, (1, 2))[:, :96]])
    b.run(3)
    before = [g.cpu().numpy() for g in b.get_phi()]
    m = b.run(0)
    assert m.shape == (0, 2, 3)
    assert all(np.array_equal(x, g.cpu().numpy()) for x, g in zip(before, b.get_phi()))
    with pytest.raises(N.LbmError) as e:
        b.run(-1, moments=False)
    assert e.value.status == N.LBM_E_ARG
    assert np.isfinite(b.run(2)).all()
    b.close()
