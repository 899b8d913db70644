"""Walls on the x faces (D2Q9 and D3Q15) and the z faces (D3Q15) of the oracle.

The paper's wall rule (Sec. 3.2) is written for walls normal to y. The lattices
are symmetric under an exchange of two axes: D2Q9 maps onto itself under
x <-> y (populations 1 <-> 2, 3 <-> 4, 6 <-> 8; the moment rows j_x <-> j_y,
q_x <-> q_y, and p_xx = e_x^2 - e_y^2 changes sign, which a diagonal rate does
not see), D3Q15 under y <-> z and x <-> y (the stress rows with equal rates map
into each other). So a run with walls on the x (or z) faces must equal, node for
node, the run with the same walls on the y faces of the grid with those two axes
exchanged (D, u, phi permuted alike). That pins the x and z walls against the y
walls, which Tables 3-5 pin (tests/test_oracle_taylor_aris.py). Edges where two
wall faces meet are checked by the same exchange (walls of kinds K1 on x and K2
on y equal K2 on x and K1 on y, transposed), by exact conservation under
bounce-back on every face, and by a pull-form evaluation of the rules written
here on a tiny box.
"""
import numpy as np
import pytest

from paper_1404_2363_gb300 import workloads as W


def _fields2(nx, ny, seed):
    g = np.random.default_rng(seed)
    phi = 0.5 + g.random((ny, nx))
    u = g.uniform(-0.05, 0.05, (2, ny, nx))
    return phi, u


def _run2(O, phi, u, D, steps, bcx=(0, 0), bcy=(0, 0)):
    ny, nx = phi.shape
    p = O.Params(nx=nx, ny=ny, A=O.A_from_D(D), bc_lo=bcy[0], bc_hi=bcy[1], bcx_lo=bcx[0], bcx_hi=bcx[1])
    return O.run(p, phi.reshape(-1), steps, u=u.reshape(2, -1)).reshape(ny, nx)


def _swap2(phi, u, D):
    """x <-> y: transposed fields, exchanged velocity components, D' = P D P."""
    P = np.array([[0, 1], [1, 0]])
    return phi.T.copy(), np.stack([u[1].T, u[0].T]).copy(), P @ D @ P


@pytest.mark.parametrize("kind", ["NOFLUX_NODE", "BOUNCEBACK"])
def test_x_walls_equal_y_walls_on_the_transposed_grid(O, kind):
    k = getattr(O, kind)
    phi, u = _fields2(13, 9, 1)
    D = W.D_ANISO
    got = _run2(O, phi, u, D, 60, bcx=(k, k))
    ps, us, Ds = _swap2(phi, u, D)
    want = _run2(O, ps, us, Ds, 60, bcy=(k, k)).T
    assert np.abs(got - want).max() < 1e-13
    # and the walls do act: the periodic run differs
    assert np.abs(got - _run2(O, phi, u, D, 60)).max() > 1e-4


@pytest.mark.parametrize("kx,ky", [("NOFLUX_NODE", "BOUNCEBACK"), ("BOUNCEBACK", "BOUNCEBACK"),
                                   ("NOFLUX_NODE", "NOFLUX_NODE"), ("BOUNCEBACK", "NOFLUX_NODE")])
def test_box_edges_are_symmetric_under_axis_exchange(O, kx, ky):
    a, b = getattr(O, kx), getattr(O, ky)
    phi, u = _fields2(11, 8, 2)
    D = W.D_ANISO
    got = _run2(O, phi, u, D, 40, bcx=(a, a), bcy=(b, b))
    ps, us, Ds = _swap2(phi, u, D)
    want = _run2(O, ps, us, Ds, 40, bcx=(b, b), bcy=(a, a)).T
    assert np.abs(got - want).max() < 1e-13


def test_bounceback_box_conserves_mass(O):
    """Halfway bounce-back on all four faces (and all six in 3D) returns every
    population that would leave: sum phi is constant to round-off, with a
    velocity that has components normal to every wall."""
    phi, u = _fields2(12, 10, 3)
    p = O.Params(nx=12, ny=10, A=O.A_from_D(W.D_ANISO), bc_lo=O.BOUNCEBACK, bc_hi=O.BOUNCEBACK,
                 bcx_lo=O.BOUNCEBACK, bcx_hi=O.BOUNCEBACK)
    f = O.init_eq(p, phi.reshape(-1), u.reshape(2, -1))
    m0 = f.sum()
    for _ in range(50):
        f = O.step(p, f, u.reshape(2, -1))
    assert abs(f.sum() - m0) / m0 < 1e-13
    g = np.random.default_rng(4)
    n = (7, 6, 5)
    phi3 = 0.5 + g.random(n[::-1])
    u3 = g.uniform(-0.05, 0.05, (3,) + n[::-1])
    p3 = O.default_params_3d(nx=n[0], ny=n[1], nz=n[2], A=O.A_from_D(np.diag([0.02, 0.03, 0.04]), q=15,
                                                                   alpha1=-1.2, alpha2=192.0),
                             bc_lo=O.BOUNCEBACK, bc_hi=O.BOUNCEBACK, bcx_lo=O.BOUNCEBACK, bcx_hi=O.BOUNCEBACK,
                             bcz_lo=O.BOUNCEBACK, bcz_hi=O.BOUNCEBACK)
    f = O.init_eq(p3, phi3.reshape(-1), u3.reshape(3, -1))
    m0 = f.sum()
    for _ in range(30):
        f = O.step(p3, f, u3.reshape(3, -1))
    assert abs(f.sum() - m0) / m0 < 1e-13


def test_box_rules_in_pull_form_on_a_tiny_grid(O):
    """Brute force on a 4 x 3 box (x walls Neumann, y walls bounce-back): the
    oracle's push step equals the rules evaluated here in pull form. Pull
    f_i(x) = f'_i(x - e_i); a source beyond a bounce-back face gives
    f'_opp(i)(x); then a population whose source lies beyond Neumann faces takes
    the value of the population reflected in those axes."""
    nx, ny = 4, 3
    phi, u = _fields2(nx, ny, 5)
    p = O.Params(nx=nx, ny=ny, A=O.A_from_D(W.D_ANISO), bc_lo=O.BOUNCEBACK, bc_hi=O.BOUNCEBACK,
                 bcx_lo=O.NOFLUX_NODE, bcx_hi=O.NOFLUX_NODE)
    uf = u.reshape(2, -1)
    f = O.init_eq(p, phi.reshape(-1), uf) + 0.01 * np.random.default_rng(6).standard_normal(9 * nx * ny)
    e = O.tables(p)[0]
    fr = f.reshape(9, ny, nx)
    post = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            post[:, y, x] = O.collide_node(p, fr[:, y, x], uf[:, y * nx + x])
    opp = [int(np.where((e == -e[i]).all(axis=1))[0][0]) for i in range(9)]
    want = np.zeros_like(post)
    nfmask = np.zeros((9, ny, nx), dtype=int)
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                sx, sy = x - e[i, 0], y - e[i, 1]
                out_x, out_y = not 0 <= sx < nx, not 0 <= sy < ny
                if out_y:                       # beyond a bounce-back face
                    want[i, y, x] = post[opp[i], y, x]
                elif out_x:                     # beyond a Neumann face only
                    want[i, y, x] = np.nan
                else:
                    want[i, y, x] = post[i, sy, sx]
                nfmask[i, y, x] = 1 if out_x else 0
    pulled = want.copy()
    for i in range(9):
        j = int(np.where((e[:, 0] == -e[i, 0]) & (e[:, 1] == e[i, 1]))[0][0])   # reflected in x
        for y in range(ny):
            for x in range(nx):
                if nfmask[i, y, x]:
                    want[i, y, x] = pulled[j, y, x]
    got = O.step(p, f, uf).reshape(9, ny, nx)
    assert not np.isnan(want).any()
    assert np.abs(got - want).max() < 1e-15


def _fields3(n, seed):
    g = np.random.default_rng(seed)
    phi = 0.5 + g.random(n[::-1])
    u = g.uniform(-0.05, 0.05, (3,) + n[::-1])
    return phi, u


def _run3(O, phi, u, D, steps, bc):
    nz, ny, nx = phi.shape
    p = O.default_params_3d(nx=nx, ny=ny, nz=nz, A=O.A_from_D(D, q=15, alpha1=-1.2, alpha2=192.0), **bc)
    return O.run(p, phi.reshape(-1), steps, u=u.reshape(3, -1)).reshape(nz, ny, nx)


@pytest.mark.parametrize("kind", ["NOFLUX_NODE", "BOUNCEBACK"])
@pytest.mark.parametrize("axis", ["x", "z"])
def test_d3q15_x_and_z_walls_equal_y_walls_on_the_permuted_grid(O, kind, axis):
    k = getattr(O, kind)
    n = (7, 6, 5)
    phi, u = _fields3(n, 7)
    D = np.array([[0.03, 0.005, -0.004], [0.005, 0.025, 0.003], [-0.004, 0.003, 0.035]])
    a = 2 if axis == "x" else 0                    # the axis exchanged with y (array axes: z 0, y 1, x 2)
    got = _run3(O, phi, u, D, 25, {f"bc{axis}_lo": k, f"bc{axis}_hi": k})
    perm = [0, 1, 2]
    perm[a], perm[1] = perm[1], perm[a]            # array-axis permutation
    comp = {"x": [1, 0, 2], "z": [0, 2, 1]}[axis]  # velocity components / D indices
    ps = np.transpose(phi, perm).copy()
    us = np.stack([np.transpose(u[c], perm) for c in comp]).copy()
    Ds = D[np.ix_(comp, comp)]
    want = np.transpose(_run3(O, ps, us, Ds, 25, {"bc_lo": k, "bc_hi": k}), perm)
    assert np.abs(got - want).max() < 1e-13
