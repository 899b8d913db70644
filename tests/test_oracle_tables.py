"""Pins of the oracle's lattice tables against what the paper fixes.

The oracle types M from Eq. 12 / A.2, builds e_i from Eq. 2 (D2Q9) and from
the j-rows of Eq. A.2 (D3Q15), inverts M numerically and builds S from
Eq. 31 / A.5. These tests check those tables against independent facts:
the velocity set of Eq. 2 / A.1, the Gram-Schmidt orthogonality of M,
the explicit f^eq of Eq. 17 and the moment definitions.
"""
import itertools
import math

import numpy as np
import pytest


def test_d2q9_velocities_follow_eq2(O):
    e, M, _, _ = O.tables(O.Params())
    want = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert [tuple(r[:2]) for r in e] == want
    # rows 3 and 5 of M are the x and y momentum moments (j_x, j_y)
    assert np.array_equal(M[3], e[:, 0])
    assert np.array_equal(M[5], e[:, 1])


def test_d2q9_moment_rows_are_their_definitions(O):
    """Rows of Eq. 12 as polynomials of e (c = 1): e = -4 + 3|e|^2,
    eps = 4 - 21/2 |e|^2 + 9/2 |e|^4, q_x = (-5 + 3|e|^2) e_x,
    p_xx = e_x^2 - e_y^2, p_xy = e_x e_y (Lallemand-Luo basis)."""
    e, M, _, _ = O.tables(O.Params())
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    e2 = ex * ex + ey * ey
    assert np.allclose(M[0], 1)
    assert np.allclose(M[1], -4 + 3 * e2)
    assert np.allclose(M[2], 4 - 10.5 * e2 + 4.5 * e2 * e2)
    assert np.allclose(M[4], (-5 + 3 * e2) * ex)
    assert np.allclose(M[6], (-5 + 3 * e2) * ey)
    assert np.allclose(M[7], ex * ex - ey * ey)
    assert np.allclose(M[8], ex * ey)


@pytest.mark.parametrize("q", [9, 15])
def test_M_rows_orthogonal_and_inverse(O, q):
    p = O.Params() if q == 9 else O.default_params_3d()
    _, M, Mi, _ = O.tables(p)
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.abs(M @ Mi - np.eye(q)).max() < 1e-13
    assert np.abs(Mi @ M - np.eye(q)).max() < 1e-13
    # M^-1 = M^T diag(1/|row|^2) is a consequence of orthogonality; the oracle
    # inverts numerically, so this is an independent check of its inverse.
    assert np.abs(Mi - M.T @ np.diag(1.0 / np.diag(G))).max() < 1e-14
    if q == 9:
        assert np.allclose(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    else:
        assert np.allclose(np.diag(G), [15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8])


def test_d3q15_velocity_set_is_eq_a1(O):
    e, M, _, _ = O.tables(O.default_params_3d())
    got = sorted(tuple(r) for r in e)
    want = [(0, 0, 0)]
    want += [(s, 0, 0) for s in (1, -1)] + [(0, s, 0) for s in (1, -1)] + [(0, 0, s) for s in (1, -1)]
    want += list(itertools.product((1, -1), repeat=3))
    assert got == sorted(want)
    assert tuple(e[0]) == (0, 0, 0)
    assert all(sum(abs(c) for c in e[i]) == 1 for i in range(1, 7))
    assert all(all(abs(c) == 1 for c in e[i]) for i in range(7, 15))
    ex, ey, ez = (e[:, a].astype(float) for a in range(3))
    e2 = ex * ex + ey * ey + ez * ez
    assert np.allclose(M[1], e2 - 2)                 # energy
    assert np.allclose(M[9], 3 * ex * ex - e2)        # 3 p_xx
    assert np.allclose(M[10], ey * ey - ez * ez)      # p_ww
    assert np.allclose(M[11], ex * ey)
    assert np.allclose(M[12], ey * ez)
    assert np.allclose(M[13], ex * ez)
    assert np.allclose(M[14], ex * ey * ez)


def feq_eq17(a1, a2, phi, u):
    """Eq. 17, typed independently of the oracle's M^-1 m^eq route."""
    E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    out = []
    for i, (ex, ey) in enumerate(E):
        eu = ex * u[0] + ey * u[1]
        if i == 0:
            out.append((-a1 + a2 + 4) * phi / 36)
        elif i <= 4:
            out.append((-a1 - 2 * a2 + 16 + 48 * eu) * phi / 144)
        else:
            out.append((2 * a1 + a2 + 16 + 12 * eu) * phi / 144)
    return np.array(out)


@pytest.mark.parametrize("a1,a2", [(-8.0, 8.0), (-4.0, 3.0), (2.5, -1.0)])
def test_feq_equals_eq17(O, a1, a2):
    g = np.random.default_rng(1)
    p = O.Params(alpha1=a1, alpha2=a2)
    _, M, Mi, _ = O.tables(p)
    e = O.tables(p)[0][:, :2]
    for _ in range(5):
        phi = g.uniform(0.2, 2.0)
        u = g.uniform(-0.1, 0.1, 2)
        fe = Mi @ O.meq(p, phi, u)
        assert np.allclose(fe, feq_eq17(a1, a2, phi, u), rtol=0, atol=1e-15)
        assert abs(fe.sum() - phi) < 1e-14
        assert np.allclose(e.T @ fe, phi * u, atol=1e-15)


def test_mrt_a_equilibrium_weights(O):
    """Eq. 37 in velocity space: rest 5/9, every moving link 1/18,
    convective weight 1/3 (axes) and 1/12 (diagonals)."""
    p = O.Params()
    _, _, Mi, _ = O.tables(p)
    fe0 = Mi @ O.meq(p, 1.0, [0.0, 0.0])
    assert np.allclose(fe0, [5 / 9] + [1 / 18] * 8, atol=1e-15)
    fx = Mi @ O.meq(p, 1.0, [1.0, 0.0]) - fe0
    assert np.allclose(fx, [0, 1 / 3, 0, -1 / 3, 0, 1 / 12, -1 / 12, -1 / 12, 1 / 12], atol=1e-15)


def test_d3q15_equilibrium_weights(O):
    """With alpha1 = -6/5, alpha2 = 192 (the D3Q15 reading), f^eq has rest 8/15,
    every moving link 1/30, and carries phi u as its first moment (Eq. A.3-A.4)."""
    p = O.default_params_3d()
    e, _, Mi, _ = O.tables(p)
    fe0 = Mi @ O.meq(p, 1.0, [0, 0, 0])
    assert np.allclose(fe0, [8 / 15] + [1 / 30] * 14, atol=1e-15)
    u = np.array([0.03, -0.02, 0.01])
    fe = Mi @ O.meq(p, 1.3, u)
    assert abs(fe.sum() - 1.3) < 1e-14
    assert np.allclose(e.T @ fe, 1.3 * u, atol=1e-15)
    # second moment: sum e_x^2 f^eq = phi / 3 at u = 0 (the 1/3 of Eq. A.6)
    assert abs((e[:, 0] ** 2) @ fe0 - 1 / 3) < 1e-15


def test_diffusion_factor_eq36_and_a6(O):
    assert abs(O.diffusion_factor(9, -8, 8) - 1 / 3) < 1e-15
    # with alpha2 = 4 (the standard D2Q9 weights) the modified factor vanishes
    assert abs(O.diffusion_factor(9, -8, 4)) < 1e-15
    assert abs(O.diffusion_factor(15, -6 / 5, 192) - 1 / 3) < 1e-14
    D = np.array([[0.02, 0.01], [0.01, 0.04]])
    A = O.A_from_D(D)
    assert np.allclose(np.linalg.inv(A), 3 * D + 0.5 * np.eye(2))
    assert np.allclose(O.D_from_A(A), D)
    # Eq. 44 full anisotropic: A^-1 = [[tau, tau-1/2], [tau-1/2, 4 tau - 1.5]]
    tau = 0.9
    Ainv = np.array([[tau, tau - 0.5], [tau - 0.5, 4 * tau - 1.5]])
    assert np.allclose(O.D_from_A(np.linalg.inv(Ainv)), (tau - 0.5) / 3 * np.array([[1, 1], [1, 4]]))


def test_modified_S_entries_eq31(O):
    sxx, sxy, syx, syy = 1.3, 0.2, 0.25, 1.6
    s = np.array([1.0, 1.1, 1.15, 0, 1.4, 0, 1.7, 1.2, 1.25])
    p = O.Params(A=np.array([[sxx, sxy], [syx, syy]]), s=s, tie=False)
    S = O.tables(p)[3]
    want = np.diag([1.0, 1.1, 1.15, sxx, 1.4, syy, 1.7, 1.2, 1.25])
    want[3, 4] = (sxx / 2 - 1) * 1.4
    want[3, 5] = sxy
    want[3, 6] = sxy / 2 * 1.7
    want[5, 3] = syx
    want[5, 4] = syx / 2 * 1.4
    want[5, 6] = (syy / 2 - 1) * 1.7
    assert np.array_equal(S, want)
    # unmodified (Eq. 24) for the MRT-B models
    pb = O.Params(A=p.A, s=s, tie=False, model=O.MRT_B1)
    Sb = O.tables(pb)[3]
    wb = np.diag([1.0, 1.1, 1.15, sxx, 1.4, syy, 1.7, 1.2, 1.25])
    wb[3, 5], wb[5, 3] = sxy, syx
    assert np.array_equal(Sb, wb)


def test_meq_b_models_eq38_eq39(O):
    u = np.array([0.07, -0.03])
    u2 = float(u @ u)
    for model, c2 in ((O.MRT_B1, 1.0), (O.MRT_B2, 2.0)):
        m = O.meq(O.Params(model=model), 2.0, u)
        want = 2.0 * np.array([1, -2 + 3 * u2, c2 - 3 * u2, u[0], -u[0], u[1], -u[1],
                               u[0] ** 2 - u[1] ** 2, u[0] * u[1]])
        assert np.allclose(m, want, atol=1e-15)
    m3 = O.meq(O.Params(model=O.MRT_B3, alpha1=3.0, alpha2=5.0), 2.0, u)
    assert np.allclose(m3, 2.0 * np.array([1, -2, 2, u[0], -u[0], u[1], -u[1], 0, 0]), atol=1e-15)
