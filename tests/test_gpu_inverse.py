"""The inverse-problem workload at its full size: D2Q9 MRT-A on a 1024 x 1024
periodic grid with a seeded stream-function velocity, 2000 steps under sqrt(N)
checkpointing, snapshots with N(0, 1e-3^2) noise. Recover the three entries of
D and the 64 x 64 Fourier modes of phi0 (torch L-BFGS through the hand-written
adjoint): jointly from snapshots at steps 1000 and 2000, and from the final
snapshot alone with the other unknown given (jointly, one snapshot leaves a
smaller D with a smoother phi0 as good a fit); check the gradients at that size
against central differences of the GPU forward, and on a reduced grid against
the FP64 oracle adjoint."""
import numpy as np
import pytest
import torch

from _common import Case, oracle_params, rel_l2
from paper_1404_2363_gb300 import inverse as I
from paper_1404_2363_gb300 import workloads as W
from paper_1404_2363_gb300.autograd import lbm_run
from paper_1404_2363_gb300.solver import Solver

pytestmark = pytest.mark.gpu

N, STEPS, MODES, SIGMA = 1024, 2000, 64, 1e-3


def _setup(n=N, modes=MODES):
    wl = W.inverse_workload(n, modes=modes)
    s = Solver(nx=n, ny=n)
    a = torch.from_numpy(wl["u"].astype(np.float32)).cuda()
    phi0 = torch.from_numpy(wl["phi0"].astype(np.float32)).cuda()
    return wl, s, a, phi0


def _observations(s, a, phi0_true, D_true, times, seed=20140409):
    """Noisy snapshots phi(t) + N(0, SIGMA^2) of the true run at the given steps."""
    g = np.random.default_rng(seed)
    out, t_prev, phi = [], 0, phi0_true
    with torch.no_grad():
        for t in times:
            phi = lbm_run(phi, torch.tensor(D_true), a, solver=s, nsteps=t - t_prev).clone()
            noise = torch.from_numpy(g.standard_normal((N, N)) * SIGMA).cuda()
            out.append((t, phi.to(torch.float64) + noise))
            t_prev = t
    return out


def _errors(res, D_true, phi0_true):
    D_err = np.linalg.norm(res["D"] - D_true) / np.linalg.norm(D_true)
    dev_true = I.project(phi0_true.to(torch.float64) - 1.0, MODES)
    phi_err = float(torch.linalg.norm(res["phi0"] - 1.0 - dev_true) / torch.linalg.norm(dev_true))
    return D_err, phi_err


def test_inverse_problem_two_snapshots_recovers_D_and_phi0_modes():
    """Joint recovery of D (three entries) and the 64 x 64 modes of phi0 from
    noisy snapshots at steps 1000 and 2000: D within 1 %, phi0 within 5 % in the
    mode space, misfit at the noise level."""
    wl, s, a, phi0_true = _setup()
    obs = _observations(s, a, phi0_true, wl["D"], (STEPS // 2, STEPS))
    s2 = Solver(nx=N, ny=N)
    res = I.recover([s, s2], obs, a, modes=MODES, max_iter=200)
    s.close()
    s2.close()
    D_err, phi_err = _errors(res, wl["D"], phi0_true)
    floor = 2 * N * N * SIGMA ** 2
    print(f"two snapshots: D {np.round(res['D'], 6).tolist()} (relative error {D_err:.2e}); phi0 mode-space "
          f"relative error {phi_err:.2e}; misfit {res['loss']:.4f} (noise level {floor:.4f}); "
          f"{res['evaluations']} evaluations")
    assert D_err < 1e-2
    assert phi_err < 5e-2
    assert res["loss"] < 1.01 * floor


def test_inverse_problem_final_snapshot():
    """From the final snapshot alone: with D known the 64 x 64 modes of phi0 are
    recovered (a linear least-squares problem) within 5 %; with phi0 known the
    three entries of D within 0.5 %. Fitting both together reaches the noise level
    as well, but D is not determined by one snapshot (a smaller D with a smoother
    phi0 fits as well), so only the misfit is checked there."""
    wl, s, a, phi0_true = _setup()
    obs = _observations(s, a, phi0_true, wl["D"], (STEPS,))
    floor = N * N * SIGMA ** 2
    r1 = I.recover([s], obs, a, modes=MODES, fit_D=False, D_fixed=wl["D"], max_iter=150)
    _, phi_err = _errors(r1, wl["D"], phi0_true)
    r2 = I.recover([s], obs, a, modes=MODES, fit_phi0=False, phi0_fixed=phi0_true, max_iter=60)
    D_err, _ = _errors(r2, wl["D"], phi0_true)
    r3 = I.recover([s], obs, a, modes=MODES, max_iter=150)
    s.close()
    print(f"final snapshot: phi0 modes with D known {phi_err:.2e} (misfit {r1['loss']:.4f}); D with phi0 known "
          f"{D_err:.2e} (misfit {r2['loss']:.4f}); both: D {np.round(r3['D'], 6).tolist()}, misfit "
          f"{r3['loss']:.4f} (noise level {floor:.4f})")
    assert phi_err < 5e-2 and r1["loss"] < 1.01 * floor
    assert D_err < 5e-3 and r2["loss"] < 1.01 * floor
    assert r3["loss"] < 1.01 * floor


def _smooth_weight(n):
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    return (np.cos(k * x) * np.cos(2 * k * y) + 0.5 * np.sin(3 * k * x + k * y)).astype(np.float32)


def test_full_size_gradients_against_central_differences_of_the_gpu_forward():
    """L = sum_x g(x) phi_N(x) with a smooth g: the adjoint's dL/dD and dL/dphi0
    against differences of the FP32 GPU forward, both from the deviation f of the
    workload's phi0 = 1 + f (the step is linear in phi; with the constant part the
    FP32 rounding of phi ~ 1 over 2000 steps would swamp a difference of two
    runs. The constant is not an exact fixed point here: the lattice divergence
    of the sampled velocity field is not zero, so its evolution depends on D by a
    few per cent of dL/dD). dL/dD: Richardson extrapolation of
    central differences with steps of 2.5 % and 5 % of each entry (truncation
    O(h^4)), within 1e-3 of the largest entry of the gradient (the rounding noise
    left in the difference of two FP32 runs is about 1e-5 of it); dL/dphi0 at sampled cells: L is linear in phi0, so L(f + 10 e_c) - L(f)
    = 10 dL/dphi0(c) exactly up to rounding, within 1e-4."""
    wl, s, a, phi0 = _setup()
    g = torch.from_numpy(_smooth_weight(N)).cuda()
    s.set_D(wl["D"])
    s.set_velocity(a)
    dev = (phi0 - 1.0).contiguous()
    s.forward_ckpt(dev, STEPS)
    dphi0, dD, _, _ = s.backward(g)
    dphi0 = dphi0.cpu().numpy().astype(np.float64)

    def L(D, p0):
        s.set_D(D)
        s.set_phi(p0)
        s.step(STEPS)
        return float((s.get_phi().to(torch.float64) * g.to(torch.float64)).sum())

    res = {}
    for (i, j) in ((0, 0), (0, 1), (1, 1)):
        fd = []
        for h in (2.5e-2, 5e-2):
            d = h * abs(wl["D"][i, j])
            vals = []
            for sgn in (1, -1):
                D = wl["D"].copy()
                D[i, j] += sgn * d
                if i != j:
                    D[j, i] += sgn * d
                vals.append(L(D, dev))
            fd.append((vals[0] - vals[1]) / (2 * d))
        rich = (4 * fd[0] - fd[1]) / 3
        an = dD[i, j] + (dD[j, i] if i != j else 0.0)
        print(f"dL/dD[{i}{j}]: adjoint {an:.8e}, difference {rich:.8e} (steps {fd})")
        res[(i, j)] = (an, rich)
    scale = max(abs(v[1]) for v in res.values())
    for (i, j), (an, rich) in res.items():
        assert abs(an - rich) <= 1e-3 * scale, (i, j, an, rich, scale)
    base = L(wl["D"], dev)
    for (y, x) in ((0, 0), (512, 300), (1023, 17), (250, 1000)):
        p = dev.clone()
        p[y, x] += 10.0
        fd = (L(wl["D"], p) - base) / 10.0
        print(f"dL/dphi0[{y},{x}]: adjoint {dphi0[y, x]:.8e}, difference {fd:.8e}")
        assert abs(dphi0[y, x] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(dphi0).max(), (y, x, dphi0[y, x], fd)
    s.close()


def test_reduced_grid_gradients_match_the_fp64_oracle_adjoint(O):
    """The same recipe (stream-function u, Fourier phi0, anisotropic D) on a
    96 x 96 grid for 200 steps: dL/dphi0 and dL/dD of the misfit
    L = sum (phi_N - obs)^2 from the GPU adjoint against the oracle adjoint."""
    n, steps = 96, 200
    wl = W.inverse_workload(n, modes=16)
    phi0 = wl["phi0"].astype(np.float32)
    u = wl["u"].astype(np.float32)
    obs = phi0.astype(np.float64) + 1e-3 * np.random.default_rng(3).standard_normal((n, n))
    s = Solver(nx=n, ny=n)
    s.set_D(wl["D"])
    s.set_velocity(torch.from_numpy(u).cuda())
    phiN = s.forward_ckpt(torch.from_numpy(phi0).cuda(), steps).cpu().numpy().astype(np.float64)
    g = 2.0 * (phiN - obs)
    dphi0, dD, _, _ = s.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    s.close()
    case = Case(nx=n, ny=n, D=wl["D"])
    p = oracle_params(O, case)
    gp, gD, _, _ = O.adjoint_gradients(p, phi0.astype(np.float64).reshape(-1), steps, g.reshape(-1),
                                       u=u.astype(np.float64).reshape(2, -1))
    assert rel_l2(dphi0.cpu().numpy().astype(np.float64), gp.reshape(n, n)) < 1e-5
    assert np.abs(dD - gD).max() <= 1e-4 * np.abs(gD).max()
