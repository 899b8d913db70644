"""Pins of the oracle's reverse-time (adjoint) step.

For a fixed velocity field one time step is linear in f (Eq. 11-15 with m^eq
linear in phi), f(t+1) = T f(t). The oracle's adjoint step must equal T^T:
T is assembled here column by column from the forward oracle step applied to
unit vectors (brute force). Gradients of a misfit with respect to D, u and
phi0 are then checked against central finite differences in FP64.
"""
import numpy as np
import pytest

from paper_1404_2363_gb300 import workloads as W


def assemble_T(O, p, u):
    n = p.q * p.ncell
    T = np.zeros((n, n))
    post = np.empty(n)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        T[:, j] = O.step(p, e, u, post)
    return T


@pytest.mark.parametrize("bc", ["periodic", "noflux", "bounceback"])
@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_step_is_transpose(O, bc, model):
    nx, ny = 4, 5
    kind = {"periodic": O.PERIODIC, "noflux": O.NOFLUX_NODE, "bounceback": O.BOUNCEBACK}[bc]
    p = O.Params(nx=nx, ny=ny, bc_lo=kind, bc_hi=kind, A=O.A_from_D(W.D_ANISO), model=model)
    phi, u = W.random_fields(nx, ny, seed=5)
    u = u.reshape(2, -1)
    T = assemble_T(O, p, u)
    g = np.random.default_rng(7)
    lam = g.standard_normal(9 * nx * ny)
    f = g.standard_normal(9 * nx * ny)
    got, _, _ = O.adjoint_step(p, lam, f, u)
    assert np.abs(got - T.T @ lam).max() < 1e-13
    if bc == "periodic":
        # columns of T sum to one per (i, x): mass is conserved (Eq. 15a)
        assert np.abs(T.sum(axis=0) - 1.0).max() < 1e-13


@pytest.mark.parametrize("bx", [("periodic", "periodic"), ("noflux", "bounceback")])
def test_adjoint_step_is_transpose_with_dirichlet_walls(O, bx):
    """Dirichlet walls (Sec. 3.2, wall-node phi_w) make the step affine,
    f(t+1) = T f(t) + b: the adjoint step equals T^T of its linear part, the
    constant b (from phi_w) being removed by taking differences; alone and
    meeting walls on the x faces."""
    K = {"periodic": O.PERIODIC, "noflux": O.NOFLUX_NODE, "bounceback": O.BOUNCEBACK}
    nx, ny = 4, 5
    p = O.Params(nx=nx, ny=ny, A=O.A_from_D(W.D_ANISO), bc_lo=O.DIRICHLET, bc_hi=O.DIRICHLET,
                 phi_w_lo=1.0, phi_w_hi=0.25, bcx_lo=K[bx[0]], bcx_hi=K[bx[1]])
    g = np.random.default_rng(12)
    u = g.uniform(-0.05, 0.05, (2, nx * ny))
    n = 9 * nx * ny
    post = np.empty(n)
    b = O.step(p, np.zeros(n), u, post)
    T = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        T[:, j] = O.step(p, e, u, post) - b
    assert np.abs(b).max() > 0.01            # the walls do add a constant
    lam = g.standard_normal(n)
    f = g.standard_normal(n)
    got, _, _ = O.adjoint_step(p, lam, f, u)
    assert np.abs(got - T.T @ lam).max() < 1e-12
    with pytest.raises(RuntimeError):
        O.adjoint_step(p, lam, f, u, want_du=True)   # velocity partials: not with Dirichlet


BOXES = [
    # (lattice, x faces, y faces, z faces)
    (9, ("noflux", "noflux"), ("periodic", "periodic"), None),
    (9, ("bounceback", "bounceback"), ("noflux", "noflux"), None),
    (9, ("noflux", "bounceback"), ("bounceback", "noflux"), None),
    (15, ("periodic", "periodic"), ("periodic", "periodic"), ("noflux", "bounceback")),
    (15, ("bounceback", "noflux"), ("noflux", "bounceback"), ("noflux", "noflux")),
]


@pytest.mark.parametrize("lattice,bx,by,bz", BOXES, ids=lambda v: "-".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_adjoint_step_is_transpose_with_walls_on_any_face(O, lattice, bx, by, bz):
    """Walls on the x (and z) faces, alone and meeting other walls at edges and
    corners: the adjoint step still equals T^T of the assembled forward step."""
    K = {"periodic": O.PERIODIC, "noflux": O.NOFLUX_NODE, "bounceback": O.BOUNCEBACK}
    kw = dict(bc_lo=K[by[0]], bc_hi=K[by[1]], bcx_lo=K[bx[0]], bcx_hi=K[bx[1]])
    g = np.random.default_rng(11)
    if lattice == 9:
        nx, ny = 4, 5
        p = O.Params(nx=nx, ny=ny, A=O.A_from_D(W.D_ANISO), **kw)
        u = g.uniform(-0.05, 0.05, (2, nx * ny))
        n = 9 * nx * ny
    else:
        nx, ny, nz = 3, 4, 3
        D = np.array([[0.03, 0.005, -0.004], [0.005, 0.025, 0.003], [-0.004, 0.003, 0.035]])
        p = O.default_params_3d(nx=nx, ny=ny, nz=nz, A=O.A_from_D(D, q=15, alpha1=-1.2, alpha2=192.0),
                                bcz_lo=K[bz[0]], bcz_hi=K[bz[1]], **kw)
        u = g.uniform(-0.05, 0.05, (3, nx * ny * nz))
        n = 15 * nx * ny * nz
    T = assemble_T(O, p, u)
    lam = g.standard_normal(n)
    f = g.standard_normal(n)
    got, _, _ = O.adjoint_step(p, lam, f, u)
    assert np.abs(got - T.T @ lam).max() < 1e-12
    if all(b[0] in ("bounceback", "periodic") and b[1] in ("bounceback", "periodic") for b in (bx, by, bz or bx)):
        assert np.abs(T.sum(axis=0) - 1.0).max() < 1e-12   # bounce-back conserves mass


def misfit_setup(O, nx=8, ny=7, bc="periodic", model=0):
    kind = {"periodic": O.PERIODIC, "noflux": O.NOFLUX_NODE}[bc]
    p = O.Params(nx=nx, ny=ny, bc_lo=kind, bc_hi=kind, A=O.A_from_D(W.D_ANISO), model=model)
    phi0, u = W.random_fields(nx, ny, seed=6)
    obs = np.random.default_rng(9).uniform(0.5, 1.5, nx * ny)
    return p, phi0.reshape(-1), u.reshape(2, -1), obs


def loss(O, p, phi0, u, obs, nsteps):
    phi = O.run(p, phi0, nsteps, u=u)
    return 0.5 * float(((phi - obs) ** 2).sum()), phi


@pytest.mark.parametrize("bc,model", [("periodic", 0), ("noflux", 0), ("periodic", 1), ("noflux", 2)])
def test_gradients_match_central_differences(O, bc, model):
    """MRT-B1/B2 (model 1, 2) carry u^2 terms in m^eq (Eq. 38-39) and the
    unmodified S: their velocity and D gradients take other paths."""
    nsteps = 12
    p, phi0, u, obs = misfit_setup(O, bc=bc, model=model)
    L0, phiN = loss(O, p, phi0, u, obs, nsteps)
    g_phi0, gD, g_u, _ = O.adjoint_gradients(p, phi0, nsteps, phiN - obs, u=u)
    D = W.D_ANISO.copy()
    h = 1e-6
    # dL/dD for the symmetric parametrisation (D01 = D10 move together)
    for (a, b) in ((0, 0), (0, 1), (1, 1)):
        dD = np.zeros((2, 2))
        dD[a, b] = dD[b, a] = h
        Lp = loss(O, O.Params(**{**p.__dict__, "A": O.A_from_D(D + dD)}), phi0, u, obs, nsteps)[0]
        Lm = loss(O, O.Params(**{**p.__dict__, "A": O.A_from_D(D - dD)}), phi0, u, obs, nsteps)[0]
        fd = (Lp - Lm) / (2 * h)
        an = gD[a, b] + (gD[b, a] if a != b else 0.0)
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-9, (a, b, an, fd)
    g = np.random.default_rng(11)
    for c in g.choice(p.ncell, 4, replace=False):
        e = np.zeros_like(phi0)
        e[c] = h
        fd = (loss(O, p, phi0 + e, u, obs, nsteps)[0] - loss(O, p, phi0 - e, u, obs, nsteps)[0]) / (2 * h)
        assert abs(g_phi0[c] - fd) <= 1e-6 * abs(fd) + 1e-9
        for a in range(2):
            du = np.zeros_like(u)
            du[a, c] = h
            fd = (loss(O, p, phi0, u + du, obs, nsteps)[0] - loss(O, p, phi0, u - du, obs, nsteps)[0]) / (2 * h)
            assert abs(g_u[a, c] - fd) <= 1e-6 * abs(fd) + 1e-9, (a, c, g_u[a, c], fd)
