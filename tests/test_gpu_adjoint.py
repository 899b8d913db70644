"""GPU adjoint (reverse-time kernels behind lbm_cde_backward / torch.autograd)
against the FP64 oracle adjoint and central finite differences of the oracle.

The oracle adjoint is pinned separately (tests/test_oracle_adjoint.py: it equals
the transpose of the assembled one-step matrix and matches FP64 central
differences). Here the loss is L = sum_x g(x) phi_N(x) with a fixed random g,
so both sides differentiate the same functional.
"""
import numpy as np
import pytest
import torch

from _common import Case, oracle_params, rel_l2
from paper_1404_2363_gb300.solver import Solver

pytestmark = pytest.mark.gpu


def gpu_grads(case, phi0, a, sched, g, every=0):
    s = Solver(nx=case.nx, ny=case.ny, bc=case.bc, model=case.model)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda())
    phiN = s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps, every)
    dphi0, dD, ds, da = s.backward(torch.from_numpy(g.astype(np.float32)).cuda(), want_da=a is not None)
    out = (phiN.cpu().numpy().astype(np.float64), dphi0.cpu().numpy().astype(np.float64), dD,
           None if da is None else da.cpu().numpy().astype(np.float64))
    s.close()
    return out


def oracle_grads(O, case, phi0, a, sched, g):
    p = oracle_params(O, case)
    uf = case.u_of_t(a, sched)
    gp, gD, du, _ = O.adjoint_gradients(p, phi0.astype(np.float64).reshape(-1), case.steps,
                                        g.reshape(-1), u_of_t=uf)
    da = None
    if a is not None:
        s = np.ones((case.steps, case.dim)) if sched is None else \
            sched.astype(np.float64)[np.arange(case.steps) % len(sched)]
        da = np.einsum("td,tdc->dc", s, du).reshape((case.dim,) + case.shape)
    return gp.reshape(case.shape), gD, da


CASES = [
    Case(nx=70, ny=40, steps=60),
    Case(nx=70, ny=40, steps=60, sched=False),
    Case(nx=70, ny=41, steps=60, bc=("noflux", "noflux")),
    Case(nx=70, ny=41, steps=60, bc=("bounceback", "bounceback")),
    Case(nx=64, ny=33, steps=60, bc=("noflux", "noflux"), ukind="row"),
    Case(nx=64, ny=32, steps=40, ukind="none", sched=False),
    # MRT-B1/B2: m^eq with u^2 terms (Eq. 38-39), unmodified S; MRT-B3: Eq. 37
    Case(nx=70, ny=40, steps=60, model="B1"),
    Case(nx=70, ny=41, steps=60, bc=("noflux", "noflux"), model="B2"),
    Case(nx=64, ny=33, steps=60, bc=("bounceback", "bounceback"), ukind="row", model="B1"),
    Case(nx=70, ny=40, steps=60, sched=False, model="B3"),
]


@pytest.mark.parametrize("case", CASES,
                         ids=lambda c: f"{c.model}-{c.bc[0]}-{c.ukind}-{'sched' if c.sched else 'const'}")
def test_adjoint_matches_fp64_oracle_adjoint(O, case):
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(5).standard_normal(case.shape)
    a_grad = a if case.ukind == "field" else None
    phiN, dphi0, dD, da = gpu_grads(case, phi0, a, sched, g) if case.ukind == "field" else \
        _gpu_nofield(case, phi0, a, sched, g)
    wp, wD, wa = oracle_grads(O, case, phi0, a, sched, g)
    assert rel_l2(dphi0, wp) < 1e-5
    assert np.abs(dD - wD).max() <= 1e-4 * np.abs(wD).max()
    if a_grad is not None:
        assert rel_l2(da, wa) < 1e-4


def _gpu_nofield(case, phi0, a, sched, g):
    s = Solver(nx=case.nx, ny=case.ny, bc=case.bc, model=case.model)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row")
    phiN = s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps)
    dphi0, dD, ds, _ = s.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    s.close()
    return phiN.cpu().numpy(), dphi0.cpu().numpy().astype(np.float64), dD, None


def test_gradient_D_against_central_differences(O):
    """dL/dD from the GPU adjoint vs FP64 central differences of the oracle
    (the symmetric parametrisation: D01 and D10 move together)."""
    case = Case(nx=60, ny=44, steps=80)
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(8).standard_normal(case.shape)
    _, _, dD, _ = gpu_grads(case, phi0, a, sched, g)
    uf = case.u_of_t(a, sched)
    h = 1e-6
    for (i, j) in ((0, 0), (0, 1), (1, 1)):
        vals = []
        for sgn in (1, -1):
            D = case.D.copy()
            D[i, j] += sgn * h
            if i != j:
                D[j, i] += sgn * h
            p = oracle_params(O, Case(nx=case.nx, ny=case.ny, D=D))
            phi = O.run(p, phi0.astype(np.float64).reshape(-1), case.steps, u_of_t=uf)
            vals.append(float((g.reshape(-1) * phi).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = dD[i, j] + (dD[j, i] if i != j else 0.0)
        assert abs(an - fd) <= 1e-4 * abs(fd), (i, j, an, fd)


def test_checkpoint_interval_does_not_change_gradients():
    case = Case(nx=50, ny=30, steps=45)
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(2).standard_normal(case.shape)
    ref = gpu_grads(case, phi0, a, sched, g, every=1)
    for every in (0, 7, 45, 100):
        got = gpu_grads(case, phi0, a, sched, g, every=every)
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
        assert np.array_equal(got[3], ref[3])


def test_forward_ckpt_equals_plain_forward():
    from _common import run_gpu

    case = Case(nx=80, ny=36, steps=33)
    phi0, a, sched = case.inputs()
    ref, _ = run_gpu(case, phi0, a, sched)
    got = gpu_grads(case, phi0, a, sched, np.zeros(case.shape))[0]
    assert np.array_equal(got, ref)


def test_autograd_function_and_loss_backward():
    from paper_1404_2363_gb300.autograd import lbm_run

    case = Case(nx=48, ny=40, steps=30)
    phi0, a, sched = case.inputs()
    s = Solver(nx=case.nx, ny=case.ny)
    p0 = torch.from_numpy(phi0).cuda().requires_grad_(True)
    D = torch.tensor(case.D, dtype=torch.float64, requires_grad=True)
    at = torch.from_numpy(a).cuda().requires_grad_(True)
    st = torch.from_numpy(sched).cuda()
    obs = torch.rand(case.shape, device="cuda")
    phiN = lbm_run(p0, D, at, solver=s, nsteps=case.steps, sched=st)
    loss = 0.5 * ((phiN - obs) ** 2).sum()
    loss.backward()
    g = (phiN - obs).detach().cpu().numpy().astype(np.float64)
    ref = gpu_grads(case, phi0, a, sched, g)
    assert torch.allclose(p0.grad.cpu().double(), torch.from_numpy(ref[1]), rtol=1e-5, atol=1e-6)
    assert np.allclose(D.grad.numpy(), ref[2], rtol=1e-5, atol=1e-8)
    assert torch.allclose(at.grad.cpu().double(), torch.from_numpy(ref[3]), rtol=1e-4, atol=1e-6)


def test_inverse_problem_recovers_D():
    """Reduced form of the inverse-problem workload: recover the three entries of
    D from a final snapshot with L-BFGS through the adjoint."""
    from paper_1404_2363_gb300 import workloads as W
    from paper_1404_2363_gb300.autograd import lbm_run

    n, steps = 128, 300
    g = W.rng(5)
    u = W.stream_function_velocity(n, g)
    phi0 = (1.0 + W.fourier_field(n, g, modes=16)).astype(np.float32)
    D_true = W.D_ANISO
    s = Solver(nx=n, ny=n)
    a = torch.from_numpy(u.astype(np.float32)).cuda()
    p0 = torch.from_numpy(phi0).cuda()
    with torch.no_grad():
        obs = lbm_run(p0, torch.tensor(D_true), a, solver=s, nsteps=steps).clone()
    # D = L L^T with a positive diagonal keeps every trial point SPD
    theta = torch.tensor([np.log(np.sqrt(0.03)), 0.0, np.log(np.sqrt(0.03))], dtype=torch.float64,
                         requires_grad=True)

    def D_of(th):
        l00, l10, l11 = torch.exp(th[0]), th[1], torch.exp(th[2])
        return torch.stack([torch.stack([l00 * l00, l00 * l10]),
                            torch.stack([l00 * l10, l10 * l10 + l11 * l11])])

    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=40, line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        phiN = lbm_run(p0, D_of(theta), a, solver=s, nsteps=steps)
        loss = ((phiN - obs) ** 2).sum() * 1e3
        loss.backward()
        return loss

    for _ in range(3):
        opt.step(closure)
    est = D_of(theta).detach().numpy()
    assert np.allclose(est, D_true, rtol=2e-3, atol=2e-5), est


def test_d3q15_adjoint_matches_oracle_and_fd(O):
    """The same reverse-time kernel on the D3Q15 lattice (Appendix A): dL/dphi0 and
    dL/da against the FP64 oracle adjoint, dL/dD against FP64 central differences."""
    D = np.array([[0.03, 0.004, -0.003], [0.004, 0.025, 0.002], [-0.003, 0.002, 0.035]])
    case = Case(lattice=15, nx=12, ny=10, nz=9, steps=20, D=D)
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(4).standard_normal(case.shape)
    s = Solver(lattice=15, nx=case.nx, ny=case.ny, nz=case.nz)
    s.set_D(D)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps)
    dphi0, dD, _, da = s.backward(torch.from_numpy(g.astype(np.float32)).cuda(), want_da=True)
    s.close()
    wp, _, wa = oracle_grads(O, case, phi0, a, sched, g)
    assert rel_l2(dphi0.cpu().numpy().astype(np.float64), wp) < 1e-5
    assert rel_l2(da.cpu().numpy().astype(np.float64), wa) < 1e-4
    uf = case.u_of_t(a, sched)
    h = 1e-6
    for (i, j) in ((0, 0), (0, 1), (1, 2), (2, 2)):
        vals = []
        for sgn in (1, -1):
            Dp = D.copy()
            Dp[i, j] += sgn * h
            if i != j:
                Dp[j, i] += sgn * h
            p = oracle_params(O, Case(lattice=15, nx=case.nx, ny=case.ny, nz=case.nz, D=Dp))
            phi = O.run(p, phi0.astype(np.float64).reshape(-1), case.steps, u_of_t=uf)
            vals.append(float((g.reshape(-1) * phi).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = dD[i, j] + (dD[j, i] if i != j else 0.0)
        assert abs(an - fd) <= 1e-4 * abs(fd) + 1e-7, (i, j, an, fd)


BOX_ADJ = [
    Case(nx=37, ny=29, steps=40, bc=("bounceback", "noflux"), bc_x=("noflux", "bounceback")),
    Case(nx=40, ny=30, steps=40, bc_x=("bounceback", "bounceback")),
    Case(nx=33, ny=27, steps=40, bc=("noflux", "noflux"), bc_x=("noflux", "noflux"), ukind="row"),
    Case(lattice=15, nx=12, ny=10, nz=9, steps=20, bc=("noflux", "noflux"), bc_x=("bounceback", "bounceback"),
         bc_z=("noflux", "bounceback"),
         D=np.array([[0.03, 0.004, -0.003], [0.004, 0.025, 0.002], [-0.003, 0.002, 0.035]])),
    Case(nx=37, ny=29, steps=40, bc=("bounceback", "noflux"), bc_x=("noflux", "bounceback"), model="B2"),
]


@pytest.mark.parametrize("case", BOX_ADJ,
                         ids=lambda c: f"q{c.lattice}-{c.model}-x{c.bc_x[0]}-{c.bc_x[1]}-y{c.bc[0]}-{c.ukind}")
def test_adjoint_with_walls_on_x_and_z_faces(O, case):
    """Walls on the x (and z) faces, meeting the y walls at edges and corners:
    the reverse-time kernel's wall mode 2 (each pull source found as in the
    forward box kernel, the push scattering to the address the pull read)
    against the FP64 oracle adjoint, whose walls on any face are pinned as the
    transpose of the assembled step (tests/test_oracle_adjoint.py)."""
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(8).standard_normal(case.shape)
    s = Solver(lattice=case.lattice, nx=case.nx, ny=case.ny, nz=case.nz, bc=case.bc, bc_x=case.bc_x,
               bc_z=case.bc_z or ("periodic", "periodic"), model=case.model)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row" if case.ukind == "row" else "field")
    s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps)
    want_da = case.ukind == "field"
    dphi0, dD, _, da = s.backward(torch.from_numpy(g.astype(np.float32)).cuda(), want_da=want_da)
    s.close()
    wp, wD, wa = oracle_grads(O, case, phi0, a, sched, g)
    assert rel_l2(dphi0.cpu().numpy().astype(np.float64), wp) < 1e-5
    if want_da:
        assert rel_l2(da.cpu().numpy().astype(np.float64), wa) < 1e-4
    if wD is not None:
        assert np.abs(dD - wD).max() <= 1e-4 * np.abs(wD).max()
    else:   # D3Q15: dL/dD against FP64 central differences of the oracle
        uf = case.u_of_t(a, sched)
        h = 1e-6
        for (i, j) in ((0, 0), (1, 2)):
            vals = []
            for sgn in (1, -1):
                Dp = case.D.copy()
                Dp[i, j] += sgn * h
                if i != j:
                    Dp[j, i] += sgn * h
                p = oracle_params(O, Case(lattice=15, nx=case.nx, ny=case.ny, nz=case.nz, D=Dp, bc=case.bc,
                                          bc_x=case.bc_x, bc_z=case.bc_z))
                phi = O.run(p, phi0.astype(np.float64).reshape(-1), case.steps, u_of_t=uf)
                vals.append(float((g.reshape(-1) * phi).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = dD[i, j] + (dD[j, i] if i != j else 0.0)
            assert abs(an - fd) <= 1e-4 * abs(fd) + 1e-7, (i, j, an, fd)


DIRICHLET_ADJ = [
    Case(nx=70, ny=41, steps=60, bc=("dirichlet", "dirichlet"), phi_w=(1.0, 0.25)),
    Case(nx=64, ny=33, steps=60, bc=("dirichlet", "noflux"), phi_w=(0.5, 0.0), ukind="row"),
    Case(nx=37, ny=29, steps=40, bc=("dirichlet", "dirichlet"), phi_w=(1.0, 0.25), bc_x=("noflux", "bounceback")),
]


@pytest.mark.parametrize("case", DIRICHLET_ADJ, ids=lambda c: f"{c.bc[0]}-{c.bc[1]}-x{c.bc_x[0]}-{c.ukind}")
def test_adjoint_with_dirichlet_walls(O, case):
    """Dirichlet walls (Sec. 3.2) make the step affine; the reverse-time kernels
    transpose its linear part (the fill's weights w = f^eq(1, u(k - 1)) at the
    wall node), in the y-wall mode and, with walls on the x faces too, in the box
    mode: dL/dphi0 and dL/dD against the FP64 oracle adjoint, whose Dirichlet
    transpose is pinned against the assembled step (tests/test_oracle_adjoint.py).
    Velocity gradients are not formed with Dirichlet walls (LBM_E_UNSUPPORTED)."""
    from paper_1404_2363_gb300 import _native as N

    phi0, a, sched = case.inputs()
    g = np.random.default_rng(9).standard_normal(case.shape)
    s = Solver(nx=case.nx, ny=case.ny, bc=case.bc, bc_x=case.bc_x, phi_w=case.phi_w)
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row" if case.ukind == "row" else "field")
    s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps)
    dphi0, dD, _, _ = s.backward(torch.from_numpy(g.astype(np.float32)).cuda(), want_da=False)
    if case.ukind == "field":
        with pytest.raises(N.LbmError) as e:
            s.backward(torch.from_numpy(g.astype(np.float32)).cuda(), want_da=True)
        assert e.value.status == N.LBM_E_UNSUPPORTED
    s.close()
    wp, wD, _ = oracle_grads(O, case, phi0, None, sched, g) if case.ukind == "none" else \
        _oracle_grads_nou(O, case, phi0, a, sched, g)
    assert rel_l2(dphi0.cpu().numpy().astype(np.float64), wp) < 1e-5
    assert np.abs(dD - wD).max() <= 1e-4 * np.abs(wD).max()


def _oracle_grads_nou(O, case, phi0, a, sched, g):
    p = oracle_params(O, case)
    gp, gD, _, _ = O.adjoint_gradients(p, phi0.astype(np.float64).reshape(-1), case.steps, g.reshape(-1),
                                       u_of_t=case.u_of_t(a, sched))
    return gp.reshape(case.shape), gD, None


def test_single_step_api_matches_backward():
    """lbm_cde_adjoint_step driven step by step from the host (forward states kept
    with get_state, compensated FP32 gradient accumulators) gives the same dL/dD
    and dL/da as lbm_cde_backward."""
    import ctypes

    from paper_1404_2363_gb300 import _native as N

    case = Case(nx=48, ny=36, steps=25)
    phi0, a, sched = case.inputs()
    g = np.random.default_rng(11).standard_normal(case.shape).astype(np.float32)
    s = Solver(nx=case.nx, ny=case.ny)
    s.set_D(case.D)
    s.set_velocity(torch.from_numpy(a).cuda(), torch.from_numpy(sched).cuda())
    # reference: the checkpointed reverse sweep
    s.forward_ckpt(torch.from_numpy(phi0).cuda(), case.steps)
    _, dD_ref, _, da_ref = s.backward(torch.from_numpy(g).cuda(), want_da=True)
    # the same by single steps
    s.set_phi(torch.from_numpy(phi0).cuda())
    states = [s.get_state()[0].clone()]
    for _ in range(case.steps):
        s.step(1)
        states.append(s.get_state()[0].clone())
    q, n = 9, case.nx * case.ny
    mu = torch.from_numpy(np.tile(g.reshape(1, -1), (q, 1))).cuda().contiguous()
    mu_prev = torch.empty_like(mu)
    ng = s.L.lbm_cde_adjoint_ngrad(N.LBM_D2Q9)
    acc = torch.zeros(2 * ng, device="cuda", dtype=torch.float32)
    da = torch.zeros((2, n), device="cuda", dtype=torch.float32)
    for k in range(case.steps, 0, -1):
        st = s.L.lbm_cde_adjoint_step(s.h, k, mu.data_ptr(), mu_prev.data_ptr(), states[k - 1].data_ptr(),
                                      acc.data_ptr(), da.data_ptr())
        assert st == N.LBM_OK, s.L.lbm_cde_last_error(s.h)
        mu, mu_prev = mu_prev, mu
    s.sync()
    mu0 = mu.cpu().numpy().astype(np.float64)
    pairs = acc.cpu().numpy().astype(np.float64).reshape(ng, 2)
    gsum = np.ascontiguousarray(pairs[:, 0] + pairs[:, 1])
    dD = np.zeros((2, 2))
    st = s.L.lbm_cde_grad_rates(s.h, gsum.ctypes.data_as(N._DP), dD.ctypes.data_as(N._DP), None)
    assert st == N.LBM_OK
    s.close()
    assert np.abs(dD - dD_ref).max() <= 1e-5 * np.abs(dD_ref).max()
    # backward also adds the initial-state term of B_0 = f^eq(phi0, u(0)):
    # dL/da_d += s_d(0) phi0 sum_i mu_0,i k_i e_i,d  (k = 1/3 on the axes, 1/12 on the diagonals)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
    kk = np.array([0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 1 / 12, 1 / 12, 1 / 12, 1 / 12])
    p0 = phi0.astype(np.float64).reshape(-1)
    init = np.stack([sched[0, d] * p0 * ((kk * e)[:, None] * mu0).sum(axis=0) for d, e in enumerate((ex, ey))])
    da = da.cpu().numpy().astype(np.float64) + init
    ref = da_ref.cpu().numpy().astype(np.float64).reshape(2, -1)
    assert rel_l2(da, ref) < 1e-5


@pytest.mark.parametrize("n_grid", [2048, 14000])
def test_adjoint_64bit_offsets_window(O, n_grid):
    """Past 2^31 / (q + dim) nodes the reverse-time kernel runs with 64-bit
    offsets (D2Q9 14000 x 14000). With dL/dphi_N nonzero on a small patch only,
    every gradient comes from the nodes within nsteps of it, so a periodic
    oracle box around the patch gives the same dL/dphi0 and dL/da on the box and
    the same dL/dD. The patch straddles the periodic corner. Inputs are float32
    profiles broadcast (velocity) or multiplied (phi0) on the device, operations
    the host repeats bit for bit. (2048^2: the same with 32-bit offsets.)"""
    from paper_1404_2363_gb300 import workloads as W

    nx = ny = n_grid
    assert (11 * nx * ny >= 2 ** 31) == (n_grid > 2048)
    nsteps, ph, H = 6, 4, 4 + 6 + 6
    dev = torch.device("cuda")
    # periods of tens of nodes whatever the grid (not periodic across the seam):
    # the non-equilibrium moments stay well above the FP32 rounding of f
    k = np.arange(nx, dtype=np.float64)
    ax = (0.04 * np.sin(2 * np.pi * k / 60 + 0.4)).astype(np.float32)    # a_x(y)
    ay = (0.03 * np.cos(2 * np.pi * k / 70 + 1.1)).astype(np.float32)    # a_y(x)
    px = (1.0 + 0.3 * np.sin(2 * np.pi * k / 50)).astype(np.float32)
    py = (1.0 + 0.2 * np.cos(2 * np.pi * k / 40 + 0.3)).astype(np.float32)
    sched = W.vortex_schedule(64).astype(np.float32)
    D = W.D_ANISO
    u = torch.empty((2, ny, nx), device=dev, dtype=torch.float32)
    u[0] = torch.from_numpy(ax).to(dev)[:, None]
    u[1] = torch.from_numpy(ay).to(dev)[None, :]
    phi0 = torch.from_numpy(py).to(dev)[:, None] * torch.from_numpy(px).to(dev)[None, :]
    x0, y0 = 1, ny - 2                                   # patch centre next to the corner
    ix = np.arange(x0 - H, x0 + H + 1) % nx
    iy = np.arange(y0 - H, y0 + H + 1) % ny
    gw = np.zeros((2 * H + 1, 2 * H + 1), dtype=np.float32)
    gw[H - ph:H + ph + 1, H - ph:H + ph + 1] = np.random.default_rng(17).standard_normal((2 * ph + 1, 2 * ph + 1))
    g = torch.zeros((ny, nx), device=dev, dtype=torch.float32)
    t_iy, t_ix = torch.from_numpy(iy).to(dev), torch.from_numpy(ix).to(dev)
    g[t_iy[:, None], t_ix[None, :]] = torch.from_numpy(gw).to(dev)

    s = Solver(nx=nx, ny=ny)
    s.set_D(D)
    s.set_velocity(u, torch.from_numpy(sched).to(dev))
    s.forward_ckpt(phi0, nsteps)
    dphi0, dD, _, da = s.backward(g, want_da=True)
    got_p = dphi0[t_iy[:, None], t_ix[None, :]].cpu().numpy().astype(np.float64)
    got_a = da[:, t_iy[:, None], t_ix[None, :]].cpu().numpy().astype(np.float64)
    s.close()

    n = 2 * H + 1
    wphi = np.multiply.outer(py[iy], px[ix]).astype(np.float64).reshape(-1)
    wa = np.stack([np.broadcast_to(ax[iy][:, None], (n, n)), np.broadcast_to(ay[ix][None, :], (n, n))])
    wa = wa.astype(np.float64).reshape(2, -1)
    sc = sched.astype(np.float64)
    p = O.Params(nx=n, ny=n, A=O.A_from_D(D))
    gp, gD, du, _ = O.adjoint_gradients(p, wphi, nsteps, gw.astype(np.float64).reshape(-1),
                                        u_of_t=lambda t: wa * sc[t % len(sc)][:, None])
    st = sc[np.arange(nsteps) % len(sc)]
    want_a = np.einsum("td,tdc->dc", st, du).reshape(2, n, n)
    assert rel_l2(got_p, gp.reshape(n, n)) < 1e-5
    assert rel_l2(got_a, want_a) < 1e-4
    assert np.abs(dD - gD).max() <= 1e-4 * np.abs(gD).max()
