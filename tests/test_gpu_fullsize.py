"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark uses, on outputs the oracle can compute one by
one: a window of half-width h around a sample point, run as its own periodic
box for n steps, is exact on its central (h - n - 1)-wide patch because
populations move one node per step."""
import numpy as np
import pytest
import torch

from _common import rel_l2
from paper_1404_2363_gb300 import workloads as W
from paper_1404_2363_gb300.solver import Solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 2e-3), ("bf16", 2e-3)])
def test_vortex_4096_windows(O, storage, tol):
    N, tau, nsteps, half = 4096, 1.0, 24, 40
    wl = W.vortex_workload(N, tau)
    s = Solver(nx=N, ny=N, storage=storage)
    s.set_D(wl["D"])
    a = wl["a"].astype(np.float32)
    sched = W.vortex_schedule(2000).astype(np.float32)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    # the hill plus a background, so that windows at the periodic seam carry signal
    p0 = (wl["phi0"] + 0.1).astype(np.float32)
    s.set_phi(torch.from_numpy(p0).cuda())
    s.step(nsteps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.close()
    keep = half - nsteps - 1
    n = 2 * half + 1
    g = np.random.default_rng(3)
    pts = [(0, 0), (N - 1, 17), (N // 2, N // 2)] + [tuple(g.integers(0, N, 2)) for _ in range(3)]
    for x0, y0 in pts:
        ix = np.arange(x0 - half, x0 + half + 1) % N
        iy = np.arange(y0 - half, y0 + half + 1) % N
        wa = a.astype(np.float64)[:, iy][:, :, ix].reshape(2, -1)
        p = O.Params(nx=n, ny=n, A=O.A_from_D(wl["D"]))
        sc = sched.astype(np.float64)
        want = O.run(p, p0.astype(np.float64)[np.ix_(iy, ix)].reshape(-1), nsteps,
                     u_of_t=lambda t: wa * sc[t % len(sc)][:, None]).reshape(n, n)
        c = slice(half - keep, half + keep + 1)
        assert rel_l2(got[np.ix_(iy, ix)][c, c], want[c, c]) <= tol, (x0, y0)


def test_d3q15_384_windows(O):
    N, nsteps, half = 384, 8, 14
    wl = W.d3q15_workload(N)
    s = Solver(lattice=15, nx=N, ny=N, nz=N)
    s.set_D(wl["D"])
    u = wl["u"].astype(np.float32)
    s.set_velocity(torch.from_numpy(u).cuda())
    p0 = (wl["phi0"] + 0.1).astype(np.float32)
    s.set_phi(torch.from_numpy(p0).cuda())
    s.step(nsteps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.close()
    keep = half - nsteps - 1
    n = 2 * half + 1
    for (x0, y0, z0) in [(0, 0, 0), (N // 2, N // 2, N // 2), (N - 1, 100, 7), (55, 300, 200)]:
        ix = np.arange(x0 - half, x0 + half + 1) % N
        iy = np.arange(y0 - half, y0 + half + 1) % N
        iz = np.arange(z0 - half, z0 + half + 1) % N
        wu = u.astype(np.float64)[:, iz][:, :, iy][:, :, :, ix].reshape(3, -1)
        p = O.default_params_3d(nx=n, ny=n, nz=n, A=O.A_from_D(wl["D"], q=15, alpha1=-1.2, alpha2=192.0))
        want = O.run(p, p0.astype(np.float64)[np.ix_(iz, iy, ix)].reshape(-1), nsteps, u=wu).reshape(n, n, n)
        c = slice(half - keep, half + keep + 1)
        assert rel_l2(got[np.ix_(iz, iy, ix)][c, c, c], want[c, c, c]) <= 1e-5


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 2e-3), ("bf16", 2e-3)])
def test_vortex_5000_steps_error_vs_fp64(O, storage, tol):
    """The configured length of the time-varying-velocity workload (5000 steps,
    tau = 1, full anisotropic D, Gaussian hill, vortex u(x, t)) on a 256^2 grid that
    the oracle finishes in seconds: relative L2 error of phi against FP64 stays
    within the stated tolerance for every storage form."""
    n, steps, tau = 256, 5000, 1.0
    wl = W.vortex_workload(n, tau)
    a = wl["a"].astype(np.float32)
    sched = W.vortex_schedule(2000).astype(np.float32)
    p0 = wl["phi0"].astype(np.float32)
    s = Solver(nx=n, ny=n, storage=storage)
    s.set_D(wl["D"])
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    s.set_phi(torch.from_numpy(p0).cuda())
    s.step(steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.close()
    p = O.Params(nx=n, ny=n, A=O.A_from_D(wl["D"]))
    aa = a.astype(np.float64).reshape(2, -1)
    sc = sched.astype(np.float64)
    want = O.run(p, p0.astype(np.float64).reshape(-1), steps,
                 u_of_t=lambda t: aa * sc[t % len(sc)][:, None]).reshape(n, n)
    err = rel_l2(got, want)
    print(f"{storage}: relative L2 error after {steps} steps = {err:.3e}")
    assert err <= tol
