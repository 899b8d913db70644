"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark uses, on outputs the oracle can compute one by
one: a window of half-width h around a sample point, run as its own periodic
box for n steps, is exact on its central (h - n - 1)-wide patch because
populations move one node per step."""
import numpy as np
import pytest
import torch

from _common import assert_parity, rel_l2, rel_max
from paper_1404_2363_gb300 import workloads as W
from paper_1404_2363_gb300.solver import Solver

pytestmark = pytest.mark.gpu


VORTEX_4096 = [("f32", 1e-5, None, 1.0), ("f16", 2e-3, None, 1.0), ("bf16", 2e-3, None, 1.0),
               ("f16", 2e-3, (128, 5), 1.0), ("bf16", 2e-3, (128, 5), 1.0),
               ("f16", 2e-3, (64, 6), 1.0), ("bf16", 2e-3, (128, 6), 1.0),
               ("f32", 1e-5, (128, 6), 1.0), ("f16", 2e-3, (128, 7), 1.0),
               ("bf16", 2e-3, (128, 7), 1.0), ("f16", 2e-3, (128, 8), 1.0)]
# the workload's other two relaxation times, in the launches the autotuner picks
VORTEX_4096 += [(st, tol, launch, tau) for tau in (0.6, 2.0)
                for st, tol, launch in (("f32", 1e-5, None), ("f16", 2e-3, (128, 8)), ("bf16", 2e-3, (128, 7)))]


@pytest.mark.parametrize("storage,tol,launch,tau", VORTEX_4096)
def test_vortex_4096_windows(O, storage, tol, launch, tau):
    """launch (., 5) / (., 6) / (128, 7 or 8): the node-pair, node-quad and
    TMA-staged kernels; bench.py times the autotuner's choice among them."""
    N, nsteps, half = 4096, 24, 40
    wl = W.vortex_workload(N, tau)
    s = Solver(nx=N, ny=N, storage=storage)
    if launch:
        s.set_launch(*launch)
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
        assert_parity(got[np.ix_(iy, ix)][c, c], want[c, c], tol, (x0, y0))


D3_384 = [("f32", 1e-5, None), ("f16", 2e-3, (64, 5)), ("bf16", 2e-3, (192, 5)), ("bf16", 2e-3, (128, 1)),
          ("f16", 2e-3, (256, 9)), ("bf16", 2e-3, (256, 9)), ("bf16", 2e-3, (128, 9))]


def _launch_id(v):
    return f"{v[0]}x{v[1]}" if isinstance(v, tuple) else "auto"


@pytest.mark.parametrize("storage,tol,launch", D3_384, ids=[f"{s}-{_launch_id(l)}" for s, _, l in D3_384])
def test_d3q15_384_windows(O, storage, tol, launch):
    """launch (., 5): the D3Q15 node-pair kernel of the 16-bit forms; (., 9) the
    z-walk kernel (bench.py times the autotuner's choice among them); (., 1) the
    one-node kernel."""
    N, nsteps, half = 384, 8, 14
    wl = W.d3q15_workload(N)
    s = Solver(lattice=15, nx=N, ny=N, nz=N, storage=storage)
    if launch:
        s.set_launch(*launch)
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
        assert_parity(got[np.ix_(iz, iy, ix)][c, c, c], want[c, c, c], tol, (x0, y0, z0))


D3_1000 = [("f32", None), ("f16", (64, 5)), ("bf16", (64, 5)), ("f16", (64, 1)), ("bf16", (64, 1)),
           ("f16", (256, 9)), ("bf16", (256, 9))]


@pytest.mark.parametrize("storage,launch", D3_1000, ids=[f"{s}-{_launch_id(l)}" for s, l in D3_1000])
def test_d3q15_1000_steps_error_vs_fp64(O, storage, launch):
    """The D3Q15 workload's recipe (random rotated anisotropic D, divergence-free
    random u, Gaussian hill) on a 48^3 grid (64 x 48 x 48 for the z-walk
    kernel's 64-column tiles) for 1000 steps: relative L2 error of phi against
    FP64 and the change of the total (conserved exactly by the scheme) stay within
    the bounds of the D2Q9 5000-step test."""
    n, steps = 48, 1000
    nx = 64 if launch and launch[1] == 9 else n
    wl = W.d3q15_workload(n, shape=(nx, n, n))
    u = wl["u"].astype(np.float32)
    p0 = wl["phi0"].astype(np.float32)
    s = Solver(lattice=15, nx=nx, ny=n, nz=n, storage=storage)
    if launch:
        s.set_launch(*launch)
    s.set_D(wl["D"])
    s.set_velocity(torch.from_numpy(u).cuda())
    s.set_phi(torch.from_numpy(p0).cuda())
    s.step(steps)
    got = s.get_phi().cpu().numpy().astype(np.float64)
    s.close()
    p = O.default_params_3d(nx=nx, ny=n, nz=n, A=O.A_from_D(wl["D"], q=15, alpha1=-1.2, alpha2=192.0))
    want = O.run(p, p0.astype(np.float64).reshape(-1), steps,
                 u=u.astype(np.float64).reshape(3, -1)).reshape(n, n, nx)
    err = rel_l2(got, want)
    mass = abs(got.sum() - p0.astype(np.float64).sum()) / p0.astype(np.float64).sum()
    emax = rel_max(got, want)
    print(f"D3Q15 {storage} {launch}: relative L2 error after {steps} steps = {err:.3e}, per-element {emax:.3e}, "
          f"mass change {mass:.2e}")
    assert err <= {"f32": 1e-5, "f16": 1e-4, "bf16": 2e-3}[storage]
    assert emax <= {"f32": 1e-5, "f16": 1e-4, "bf16": 2e-3}[storage]
    assert mass <= {"f32": 1e-6, "f16": 1e-5, "bf16": 2e-4}[storage]


VORTEX_5000 = [("f32", 1e-5, None, 1.0), ("f16", 2e-3, None, 1.0), ("bf16", 2e-3, None, 1.0),
               ("f16", 2e-3, (64, 5), 1.0), ("bf16", 2e-3, (64, 5), 1.0),
               ("f16", 2e-3, (64, 6), 1.0), ("bf16", 2e-3, (64, 6), 1.0),
               ("f16", 2e-3, (128, 7), 1.0), ("bf16", 2e-3, (128, 7), 1.0),
               ("f16", 2e-3, (128, 8), 1.0)]
VORTEX_5000 += [(st, tol, launch, tau) for tau in (0.6, 2.0)
                for st, tol, launch in (("f32", 1e-5, None), ("f16", 2e-3, (128, 8)), ("bf16", 2e-3, (128, 7)))]


@pytest.mark.parametrize("storage,tol,launch,tau", VORTEX_5000)
def test_vortex_5000_steps_error_vs_fp64(O, storage, tol, launch, tau):
    """The configured length of the time-varying-velocity workload (5000 steps,
    tau in {0.6, 1, 2}, full anisotropic D of Eq. 44, Gaussian hill, vortex
    u(x, t)) on a 256^2 grid that the oracle finishes in seconds: relative L2 and
    per-element errors of phi against FP64 stay within the stated tolerance for
    every storage form. At tau = 0.6, A^-1 of Eq. 44 is closest to I/2 and the
    offsets of the 16-bit forms are largest relative to f^eq."""
    n, steps = 256, 5000
    wl = W.vortex_workload(n, tau)
    a = wl["a"].astype(np.float32)
    sched = W.vortex_schedule(2000).astype(np.float32)
    p0 = wl["phi0"].astype(np.float32)
    s = Solver(nx=n, ny=n, storage=storage)
    if launch:
        s.set_launch(*launch)
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
    err, emax = assert_parity(got, want, tol, (storage, launch, tau))
    # periodic: the total is conserved exactly by the scheme (and by the oracle);
    # a systematic FP32 imbalance between the 16-bit decode and store would make
    # it drift by a fixed fraction per step (3e-8 per step before the rest offset
    # carried -phi eps0). BF16's 8-bit mantissa leaves a drift of about 1.3e-4 over
    # the 5000 steps at tau = 1, which is almost all of its error. The rounding of
    # the offsets grows with them, i.e. with tau (slower relaxation, larger
    # non-equilibrium parts): at tau = 2 the measured drifts are 5.8e-5 (FP16) and
    # 2.5e-4 (BF16), still well inside the phi tolerance; at tau = 0.6 they are
    # below 3e-5.
    mass = abs(got.sum() - p0.astype(np.float64).sum()) / p0.astype(np.float64).sum()
    print(f"{storage} {launch} tau={tau}: relative L2 error after {steps} steps = {err:.3e}, "
          f"per-element {emax:.3e}, mass change {mass:.2e}")
    assert mass <= {"f32": 1e-6, "f16": 1e-5 if tau < 2 else 1e-4, "bf16": 2e-4 if tau < 2 else 5e-4}[storage]


@pytest.mark.parametrize("mode,tile", [("per_step", 8), ("persistent", 8), ("persistent", 0)])
def test_taylor_aris_batch_64_windows(O, mode, tile):
    """The 64-channel Taylor-Aris workload of bench.py at full size, in both batch
    modes: column windows of three channels (all rows, walls included) run by the
    oracle as channels of their own are exact on their central columns."""
    from paper_1404_2363_gb300.batch import Batch, mean_velocity, poiseuille_row

    chans = W.taylor_aris_batch(64)
    descs, phis = [], []
    for c in chans:
        u = poiseuille_row(c.ny, c.U)
        descs.append({"nx": c.nx, "ny": c.ny, "D": np.eye(2) * c.alpha, "u_row": u,
                      "s": [1.0, 1.1, 1.1, None, 1 / c.tau, None, 1 / c.tau, 1.2, 1.2], "tie": False,
                      "x_ref0": 0.2 * c.nx, "x_ref_velocity": mean_velocity(u)})
        phis.append(c.phi0().astype(np.float32) + 0.05)
    nsteps, half = 20, 30
    b = Batch(descs, mode=mode, tile_rows=tile, graph_steps=16)
    b.set_phi(phis)
    b.run(nsteps, moments=False)
    got = [g.cpu().numpy().astype(np.float64) for g in b.get_phi()]
    b.close()
    keep = half - nsteps - 1
    n = 2 * half + 1
    for i in (0, 31, 63):
        c, d = chans[i], descs[i]
        for x0 in (int(0.2 * c.nx), c.nx - 3):
            ix = np.arange(x0 - half, x0 + half + 1) % c.nx
            s = [1.0, 1.1, 1.1, 0.0, 1 / c.tau, 0.0, 1 / c.tau, 1.2, 1.2]
            p = O.Params(nx=n, ny=c.ny, bc_lo=O.NOFLUX_NODE, bc_hi=O.NOFLUX_NODE,
                         A=O.A_from_D(np.eye(2) * c.alpha), s=s, tie=False)
            u = np.zeros((2, c.ny, n))
            u[0] = d["u_row"][0].astype(np.float64)[:, None]
            want = O.run(p, phis[i].astype(np.float64)[:, ix].reshape(-1), nsteps,
                         u=u.reshape(2, -1)).reshape(c.ny, n)
            cs = slice(half - keep, half + keep + 1)
            assert rel_l2(got[i][:, ix][:, cs], want[:, cs]) <= 1e-5, (i, x0)


def _separable(n, seed, lo, hi):
    """A float32 profile of length n (seeded, smooth)."""
    g = np.random.default_rng(seed)
    k = np.arange(n, dtype=np.float64)
    v = lo + (hi - lo) * 0.5 * (1.0 + np.sin(2.0 * np.pi * k / n * g.integers(1, 5) + g.uniform(0, 6.28)))
    return v.astype(np.float32)


WIDE = [(9, "f32", (256, 1)), (9, "f32", (128, 2)), (9, "bf16", (256, 1)), (9, "f16", (128, 2)),
        (15, "f32", (64, 2)), (15, "bf16", (128, 1))]


@pytest.mark.parametrize("lattice,storage,launch", WIDE, ids=[f"q{q}-{s}-{_launch_id(l)}" for q, s, l in WIDE])
def test_64bit_offsets_windows(O, lattice, storage, launch):
    """Grids past 2^31 / (q + 3) nodes (D2Q9 16384 x 11008, D3Q15 512 x 512 x 456)
    run the step kernels with 64-bit offsets; the launch shapes with 32-bit
    offsets are refused there. The fields are built on the device from float32
    profiles by broadcasts (velocity) and products (phi0), float32 operations
    the host repeats bit for bit, so that oracle windows get the same inputs."""
    from paper_1404_2363_gb300 import _native as N

    dims = (16384, 11008, 1) if lattice == 9 else (512, 512, 456)
    nx, ny, nz = dims
    dim = 2 if lattice == 9 else 3
    ncell = nx * ny * nz
    assert (lattice + 3) * ncell >= 2 ** 31
    nsteps, half = (10, 24) if lattice == 9 else (5, 12)
    prof = [_separable(n, 40 + i, -0.04, 0.04) for i, n in enumerate((ny, nx, nz))]   # a_x(y), a_y(x), a_z(.)
    pphi = [_separable(n, 50 + i, 0.6, 1.4) for i, n in enumerate((nx, ny, nz))]
    sched = W.vortex_schedule(64).astype(np.float32)
    if dim == 3:
        sched = np.concatenate([sched, sched[:, :1]], axis=1)
    dev = torch.device("cuda")
    px, py, pz = (torch.from_numpy(v).to(dev) for v in pphi)
    shape = (ny, nx) if dim == 2 else (nz, ny, nx)
    s = Solver(lattice=lattice, nx=nx, ny=ny, nz=nz, storage=storage)
    with pytest.raises(N.LbmError):
        s.set_launch(128, 5 if storage != "f32" else 6)
    s.set_launch(*launch)
    D = W.D_eq44_full(1.0) if dim == 2 else np.diag([0.03, 0.02, 0.04])
    s.set_D(D)
    u = torch.empty((dim,) + shape, device=dev, dtype=torch.float32)
    if dim == 2:
        u[0] = torch.from_numpy(prof[0]).to(dev)[:, None]      # a_x depends on y
        u[1] = torch.from_numpy(prof[1]).to(dev)[None, :]      # a_y depends on x
        phi0 = py[:, None] * px[None, :]
    else:
        u[0] = torch.from_numpy(prof[0]).to(dev)[None, :, None]
        u[1] = torch.from_numpy(prof[1]).to(dev)[None, None, :]
        u[2] = torch.from_numpy(prof[2][:nz]).to(dev)[:, None, None]
        phi0 = (pz[:, None, None] * py[None, :, None]) * px[None, None, :]
    s.set_velocity(u, torch.from_numpy(sched).to(dev))
    s.set_phi(phi0)
    del u, phi0
    s.step(nsteps)
    got = s.get_phi()
    keep = half - nsteps - 1
    n = 2 * half + 1
    c = slice(half - keep, half + keep + 1)
    sc = sched.astype(np.float64)
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2 + 3, ny // 3, nz // 2)]
    for x0, y0, z0 in pts:
        ix = np.arange(x0 - half, x0 + half + 1) % nx
        iy = np.arange(y0 - half, y0 + half + 1) % ny
        if dim == 2:
            w_phi = np.multiply.outer(pphi[1][iy], pphi[0][ix]).astype(np.float64)
            wa = np.stack([np.broadcast_to(prof[0][iy][:, None], (n, n)),
                           np.broadcast_to(prof[1][ix][None, :], (n, n))]).astype(np.float64).reshape(2, -1)
            p = O.Params(nx=n, ny=n, A=O.A_from_D(D))
            sub = got[torch.from_numpy(iy).to(dev)][:, torch.from_numpy(ix).to(dev)]
        else:
            iz = np.arange(z0 - half, z0 + half + 1) % nz
            w_phi = np.multiply.outer(np.multiply.outer(pphi[2][iz], pphi[1][iy]), pphi[0][ix]).astype(np.float64)
            wa = np.stack([np.broadcast_to(prof[0][iy][None, :, None], (n, n, n)),
                           np.broadcast_to(prof[1][ix][None, None, :], (n, n, n)),
                           np.broadcast_to(prof[2][iz][:, None, None], (n, n, n))]).astype(np.float64).reshape(3, -1)
            p = O.default_params_3d(nx=n, ny=n, nz=n, A=O.A_from_D(D, q=15, alpha1=-1.2, alpha2=192.0))
            t_iz, t_iy, t_ix = (torch.from_numpy(v).to(dev) for v in (iz, iy, ix))
            sub = got[t_iz][:, t_iy][:, :, t_ix]
        want = O.run(p, w_phi.reshape(-1), nsteps,
                     u_of_t=lambda t: wa * sc[t % len(sc)][:, None]).reshape(w_phi.shape)
        g = sub.cpu().numpy().astype(np.float64)
        win = (c, c) if dim == 2 else (c, c, c)
        assert_parity(g[win], want[win], 1e-5 if storage == "f32" else 2e-3, (x0, y0, z0))
    s.close()
