"""Pins of the oracle's full time step (collision + push streaming + walls).

Exact facts used (lattice units, dt = dx = 1):
* periodic domains conserve sum(phi) (m_0 is conserved, Eq. 15a; Eq. 5 permutes);
* with a constant u and an equilibrium start the centroid moves by exactly u per
  step (the summed non-equilibrium moments stay zero under Eq. 13);
* the second spatial moments grow by exactly 2 D per step once the kinetic
  transient has decayed, where D is Eq. 36's tensor. For MRT-A this holds with
  u != 0 as well (no deviation term, Eq. 36), while MRT-B3 (Eq. 29) shows the
  deviation term;
* the Sec. 3.2 wall rule copies mirror populations at the wall nodes;
* halfway bounce-back conserves sum(phi) exactly.
"""
import numpy as np
import pytest

from paper_1404_2363_gb300 import workloads as W


def moments2d(phi, nx, ny):
    phi = phi.reshape(ny, nx)
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float), indexing="xy")
    m0 = phi.sum()
    cx, cy = (X * phi).sum() / m0, (Y * phi).sum() / m0
    dx, dy = X - cx, Y - cy
    C = np.array([[(dx * dx * phi).sum(), (dx * dy * phi).sum()],
                  [(dx * dy * phi).sum(), (dy * dy * phi).sum()]]) / m0
    return m0, np.array([cx, cy]), C


def test_periodic_conservation(O):
    phi0, u = W.random_fields(24, 20, seed=1)
    p = O.Params(nx=24, ny=20, A=O.A_from_D(W.D_ANISO))
    f = O.init_eq(p, phi0, u.reshape(2, -1))
    s0 = f.sum()
    for _ in range(50):
        f = O.step(p, f, u.reshape(2, -1))
    assert abs(f.sum() - s0) / s0 < 1e-13


def test_uniform_state_is_steady(O):
    p = O.Params(nx=8, ny=6, A=O.A_from_D(W.D_ANISO))
    u = np.tile(np.array([[0.03], [-0.04]]), (1, 48))
    f0 = O.init_eq(p, np.full(48, 0.7), u)
    f = f0
    for _ in range(5):
        f = O.step(p, f, u)
    assert np.abs(f - f0).max() < 1e-15


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_constant_velocity_drift_is_exact(O, model):
    n = 64
    u = np.array([0.05, -0.03])
    p = O.Params(nx=n, ny=n, A=O.A_from_D(W.D_ANISO), model=model)
    phi0 = W.gaussian_phi0(n, n, 4.0).reshape(-1)
    uf = np.tile(u[:, None], (1, n * n))
    f = O.init_eq(p, phi0, uf)
    _, c0, _ = moments2d(O.phi_of(p, f), n, n)
    for t in range(1, 41):
        f = O.step(p, f, uf)
        _, c, _ = moments2d(O.phi_of(p, f), n, n)
        assert np.allclose(c - c0, t * u, atol=1e-11)


def _growth(O, p, u, n, t0, t1, sigma=4.0, x0=None):
    phi0 = W.gaussian_phi0(n, n, sigma, x0=x0).reshape(-1)
    uf = None if u is None else np.tile(np.asarray(u)[:, None], (1, n * n))
    f = O.init_eq(p, phi0, uf)
    C = {}
    for t in range(t1 + 1):
        if t in (t0, t0 + 1, t1 - 1, t1):
            C[t] = moments2d(O.phi_of(p, f), n, n)[2]
        if t < t1:
            f = O.step(p, f, uf)
    return C[t0 + 1] - C[t0], C[t1] - C[t1 - 1]


@pytest.mark.parametrize("D", [np.diag([0.03, 0.03]), np.diag([0.015, 0.045]), W.D_ANISO])
def test_covariance_grows_by_2D_u0(O, D):
    n = 96
    p = O.Params(nx=n, ny=n, A=O.A_from_D(D))
    _, g = _growth(O, p, None, n, 200, 260)
    assert np.abs(g - 2 * D).max() < 1e-10


def test_covariance_growth_without_deviation_mrt_a(O):
    """u = (0.05, 0.05) constant: MRT-A keeps d<xx>/dt = 2D exactly (Eq. 36);
    MRT-B3, same equilibrium with the unmodified S, shows Eq. 29's deviation
    term, and MRT-B1 / B2 cancel it through their u^2 terms (Sec. 3)."""
    n = 128
    D = W.D_ANISO
    u = [0.05, 0.05]
    A = O.A_from_D(D)
    x0 = (58, 58)  # the hill is centred at t = 120 so the periodic images stay negligible
    ga = _growth(O, O.Params(nx=n, ny=n, A=A), u, n, 200, 260, x0=x0)[1]
    assert np.abs(ga - 2 * D).max() < 1e-10
    gb3 = _growth(O, O.Params(nx=n, ny=n, A=A, model=O.MRT_B3), u, n, 200, 260, x0=x0)[1]
    # deviation of Eq. 29 for constant u: -div(k dt_ (phi u)) = +k u u : grad grad phi,
    # k = (I - A/2) A^-1 = 3 D, i.e. an extra -2 * 3 D u u^T ... in the growth rate
    dev = gb3 - 2 * D
    assert np.abs(dev).max() > 1e-4
    uu = np.outer(u, u)
    want = -2.0 * (3 * D @ uu + uu @ (3 * D)) / 2
    assert np.allclose(dev, want, atol=2e-6)
    for model in (O.MRT_B1, O.MRT_B2):
        gb = _growth(O, O.Params(nx=n, ny=n, A=A, model=model), u, n, 200, 260, x0=x0)[1]
        assert np.abs(gb - 2 * D).max() < 1e-10
    # the growth above is 2 D with A = (3 D + I/2)^-1, i.e. k = 1/3, for the B models
    # whatever constants their equilibria carry (MRT-B1's u = 0 part is alpha2 = 4)
    for model, a2 in ((O.MRT_B1, 4.0), (O.MRT_B2, 8.0), (O.MRT_B3, 8.0)):
        assert O.diffusion_factor(9, -8.0, a2, model) == 1.0 / 3.0


def test_noflux_wall_rule_sec32(O):
    nx, ny = 10, 7
    phi0, u = W.random_fields(nx, ny, seed=2)
    p = O.Params(nx=nx, ny=ny, bc_lo=O.NOFLUX_NODE, bc_hi=O.NOFLUX_NODE, A=O.A_from_D(W.D_ANISO))
    f = O.step(p, O.init_eq(p, phi0, u.reshape(2, -1)), u.reshape(2, -1)).reshape(9, ny, nx)
    for a, b in ((2, 4), (5, 8), (6, 7)):       # bottom plate
        assert np.array_equal(f[a, 0], f[b, 0])
    for a, b in ((4, 2), (7, 6), (8, 5)):       # top plate
        assert np.array_equal(f[a, -1], f[b, -1])


def test_bounceback_conserves_mass(O):
    nx, ny = 12, 9
    phi0, u = W.random_fields(nx, ny, seed=3)
    u[1] = 0.0
    p = O.Params(nx=nx, ny=ny, bc_lo=O.BOUNCEBACK, bc_hi=O.BOUNCEBACK, A=O.A_from_D(W.D_ANISO))
    f = O.init_eq(p, phi0, u.reshape(2, -1))
    s0 = f.sum()
    for _ in range(30):
        f = O.step(p, f, u.reshape(2, -1))
    assert abs(f.sum() - s0) / s0 < 1e-13


def test_dirichlet_wall_value_and_linear_profile(O):
    """Wall-node Dirichlet reading: the unknown populations are f^eq(phi*, u) with
    phi* chosen so that sum f = phi_w. The wall nodes hold phi_w exactly after
    every step, and pure diffusion between phi = 1 and phi = 0 settles to a
    profile that is linear in the interior (tolerance observed, stated here)."""
    nx, ny = 4, 17
    p = O.Params(nx=nx, ny=ny, bc_lo=O.DIRICHLET, bc_hi=O.DIRICHLET, phi_w_lo=1.0, phi_w_hi=0.0,
                 A=np.eye(2) / 0.8)
    f = O.init_eq(p, np.full(nx * ny, 0.5))
    for _ in range(3000):
        f = O.step(p, f)
    phi = O.phi_of(p, f).reshape(ny, nx)
    assert np.abs(phi[0] - 1.0).max() < 1e-14
    assert np.abs(phi[-1] - 0.0).max() < 1e-14
    col = phi[:, 0]
    inner = col[2:-2]
    slope = np.diff(inner)
    assert np.abs(slope - slope.mean()).max() < 1e-10


def test_push_equals_pull_on_tiny_grid(O):
    """Brute force on a 3 x 4 periodic grid: the oracle's push-form step equals a
    pull-form evaluation written here from Eq. 5 (f_i(x) = f'_i(x - e_i))."""
    nx, ny = 3, 4
    phi0, u = W.random_fields(nx, ny, seed=4)
    p = O.Params(nx=nx, ny=ny, A=O.A_from_D(W.D_ANISO))
    uf = u.reshape(2, -1)
    f = O.init_eq(p, phi0, uf) + 0.01 * np.random.default_rng(0).standard_normal(9 * nx * ny)
    e = O.tables(p)[0]
    post = np.zeros((9, ny, nx))
    fr = f.reshape(9, ny, nx)
    for y in range(ny):
        for x in range(nx):
            post[:, y, x] = O.collide_node(p, fr[:, y, x], uf[:, y * nx + x])
    want = np.zeros_like(post)
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                want[i, y, x] = post[i, (y - e[i, 1]) % ny, (x - e[i, 0]) % nx]
    assert np.abs(O.step(p, f, uf) - want.reshape(-1)).max() < 1e-15
