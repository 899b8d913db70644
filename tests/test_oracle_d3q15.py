"""D3Q15 (Appendix A) oracle pins.

The paper leaves alpha1, alpha2 for D3Q15 open; the reading used throughout is
alpha1 = -6/5, alpha2 = 192, which makes the A.6 factor equal 1/3. With it the
covariance of a hill grows by exactly 2 D per step with D = (A^-1 - I/2)/3,
with and without a constant velocity (no deviation term, Eq. A.6).
"""
import numpy as np
import pytest

from paper_1404_2363_gb300 import workloads as W


def P3(O, n, D, **kw):
    return O.default_params_3d(nx=n, ny=n, nz=n, A=O.A_from_D(D, q=15, alpha1=-1.2, alpha2=192.0), **kw)


def hill3(n, sigma, x0):
    j = np.arange(n, dtype=float)
    Z, Y, X = np.meshgrid(j, j, j, indexing="ij")
    return np.exp(-((X - x0[0]) ** 2 + (Y - x0[1]) ** 2 + (Z - x0[2]) ** 2) / (2 * sigma ** 2))


def moments3(phi, n):
    phi = phi.reshape(n, n, n)
    j = np.arange(n, dtype=float)
    Z, Y, X = np.meshgrid(j, j, j, indexing="ij")
    m0 = phi.sum()
    xs = [X, Y, Z]
    c = np.array([(v * phi).sum() / m0 for v in xs])
    C = np.array([[((xs[a] - c[a]) * (xs[b] - c[b]) * phi).sum() / m0 for b in range(3)] for a in range(3)])
    return m0, c, C


D3 = np.array([[0.03, 0.005, -0.004], [0.005, 0.025, 0.003], [-0.004, 0.003, 0.035]])


def test_conservation_and_fixed_point(O):
    n = 10
    p = P3(O, n, D3)
    g = np.random.default_rng(2)
    phi = 0.5 + g.random(n ** 3)
    u = g.uniform(-0.05, 0.05, (3, n ** 3))
    f = O.init_eq(p, phi, u)
    s0 = f.sum()
    for _ in range(10):
        f = O.step(p, f, u)
    assert abs(f.sum() - s0) / s0 < 1e-13
    uc = np.tile(np.array([[0.02], [-0.01], [0.03]]), (1, n ** 3))
    f0 = O.init_eq(p, np.full(n ** 3, 0.9), uc)
    assert np.abs(O.step(p, f0, uc) - f0).max() < 1e-15


def test_e1_minus_e2_perturbation_eq_a5(O):
    """m - m^eq = d (0,0,0,2,-8,0,...) (columns 1, 2 of Eq. A.2); Eq. A.5 rows 3, 5, 7."""
    A = np.array([[1.4, 0.1, -0.05], [0.1, 1.3, 0.07], [-0.05, 0.07, 1.6]])
    s = np.array([1.0, 1.1, 1.15, 0, 1.25, 0, 1.35, 0, 1.45] + [1.2] * 6)
    p = O.default_params_3d(A=A, s=s, tie=False)
    _, M, Mi, _ = O.tables(p)
    u = np.array([0.01, 0.02, -0.01])
    me = O.meq(p, 1.1, u)
    d = 4e-3
    f = Mi @ me
    f[1] += d
    f[2] -= d
    mp = M @ O.collide_node(p, f, u)
    s4 = s[4]
    want = me.copy()
    want[3] = me[3] + 2 * d - A[0, 0] * 2 * d - (A[0, 0] / 2 - 1) * s4 * (-8 * d)
    want[5] = me[5] - A[1, 0] * 2 * d - (A[1, 0] / 2) * s4 * (-8 * d)
    want[7] = me[7] - A[2, 0] * 2 * d - (A[2, 0] / 2) * s4 * (-8 * d)
    want[4] = me[4] - 8 * d - s4 * (-8 * d)
    assert np.allclose(mp, want, atol=1e-15)


def test_drift_exact(O):
    """Populations move at most one node per step, so the hill (below 1e-12 beyond
    11 nodes) cannot reach the periodic seam (24 nodes away) within 12 steps."""
    n = 48
    u = np.array([0.04, -0.03, 0.02])
    p = P3(O, n, D3)
    uf = np.tile(u[:, None], (1, n ** 3))
    f = O.init_eq(p, hill3(n, 1.5, (24.0, 24.0, 24.0)).reshape(-1), uf)
    c0 = moments3(O.phi_of(p, f), n)[1]
    for t in range(1, 13):
        f = O.step(p, f, uf)
    c = moments3(O.phi_of(p, f), n)[1]
    assert np.allclose(c - c0, 12 * u, atol=1e-12)


@pytest.mark.parametrize("u", [None, (0.03, -0.02, 0.01)])
def test_covariance_grows_by_2D(O, u):
    n = 64
    p = P3(O, n, D3)
    uf = None if u is None else np.tile(np.asarray(u)[:, None], (1, n ** 3))
    x0 = (32.0, 32.0, 32.0) if u is None else (30.5, 33.0, 31.5)
    f = O.init_eq(p, hill3(n, 2.5, x0).reshape(-1), uf)
    C = {}
    for t in range(101):
        if t in (99, 100):
            C[t] = moments3(O.phi_of(p, f), n)[2]
        if t < 100:
            f = O.step(p, f, uf)
    assert np.abs((C[100] - C[99]) - 2 * D3).max() < 1e-9
