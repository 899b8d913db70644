"""Single-node collision pins (Eq. 13, 30a-30b, 31).

The oracle collides with a dense mat-vec m' = m - S (m - m^eq). These tests
check its results against the scalar relaxation formulas of Eq. 30a/30b
evaluated by hand for chosen perturbations, against the fixed point f = f^eq,
and against exact conservation of m_0.
"""
import numpy as np
import pytest

SXX, SXY, SYY = 1.45, 0.18, 1.25
RATES = np.array([1.0, 1.1, 1.1, 0, 1.3, 0, 1.6, 1.2, 1.2])


def params(O, **kw):
    kw.setdefault("A", np.array([[SXX, SXY], [SXY, SYY]]))
    kw.setdefault("s", RATES)
    kw.setdefault("tie", False)
    return O.Params(**kw)


def test_equilibrium_is_fixed_point(O):
    for model in (O.MRT_A, O.MRT_B1, O.MRT_B2, O.MRT_B3):
        p = params(O, model=model)
        _, _, Mi, _ = O.tables(p)
        u = np.array([0.04, -0.02])
        fe = Mi @ O.meq(p, 1.7, u)
        assert np.abs(O.collide_node(p, fe, u) - fe).max() < 1e-15


def test_mass_conserved_by_collision(O):
    g = np.random.default_rng(3)
    p = params(O)
    for _ in range(10):
        f = g.uniform(0, 1, 9)
        u = g.uniform(-0.1, 0.1, 2)
        assert abs(O.collide_node(p, f, u).sum() - f.sum()) < 1e-14


@pytest.mark.parametrize("delta", [1e-2, -3e-3])
def test_e1_minus_e3_perturbation_eq30(O, delta):
    """f = f^eq + delta (e_1 - e_3): m - m^eq = delta (0,0,0,2,-4,0,0,0,0) by Eq. 12.
    Eq. 30a:  m3' = m3 - sxx (2 delta) - (sxx/2 - 1) s4 (-4 delta)
    Eq. 30b:  m5' = m5 - syx (2 delta) - (syx/2) s4 (-4 delta)
    diagonal: m4' = m4 - s4 (-4 delta); all other moments stay at equilibrium."""
    p = params(O)
    _, M, Mi, _ = O.tables(p)
    u = np.array([0.03, 0.01])
    phi = 1.2
    me = O.meq(p, phi, u)
    f = Mi @ me
    f[1] += delta
    f[3] -= delta
    mp = M @ O.collide_node(p, f, u)
    s4 = RATES[4]
    want = me.copy()
    want[3] = (me[3] + 2 * delta) - SXX * 2 * delta - (SXX / 2 - 1) * s4 * (-4 * delta)
    want[5] = me[5] - SXY * 2 * delta - (SXY / 2) * s4 * (-4 * delta)
    want[4] = (me[4] - 4 * delta) - s4 * (-4 * delta)
    assert np.allclose(mp, want, atol=1e-14)


def test_e2_minus_e4_perturbation_eq30(O):
    """f = f^eq + d (e_2 - e_4): m - m^eq = d (0,0,0,0,0,2,-4,0,0)."""
    d = 5e-3
    p = params(O)
    _, M, Mi, _ = O.tables(p)
    u = np.array([-0.02, 0.05])
    me = O.meq(p, 0.8, u)
    f = Mi @ me
    f[2] += d
    f[4] -= d
    mp = M @ O.collide_node(p, f, u)
    s6 = RATES[6]
    want = me.copy()
    want[3] = me[3] - SXY * 2 * d - (SXY / 2) * s6 * (-4 * d)
    want[5] = (me[5] + 2 * d) - SYY * 2 * d - (SYY / 2 - 1) * s6 * (-4 * d)
    want[6] = (me[6] - 4 * d) - s6 * (-4 * d)
    assert np.allclose(mp, want, atol=1e-14)


def test_unmodified_S_has_no_q_coupling(O):
    """MRT-B models (Eq. 24): the same e_1 - e_3 perturbation relaxes m3 by sxx only."""
    d = 1e-2
    p = params(O, model=O.MRT_B3)
    _, M, Mi, _ = O.tables(p)
    u = np.array([0.0, 0.0])
    me = O.meq(p, 1.0, u)
    f = Mi @ me
    f[1] += d
    f[3] -= d
    mp = M @ O.collide_node(p, f, u)
    assert abs(mp[3] - (2 * d - SXX * 2 * d)) < 1e-15
    assert abs(mp[5] - (-SXY * 2 * d)) < 1e-15


def test_energy_moment_relaxes_with_s1(O):
    """A perturbation in the energy moment only: f = f^eq + d M^-1 e_1; m1 relaxes
    with s1 and nothing else moves."""
    d = 0.02
    p = params(O)
    _, M, Mi, _ = O.tables(p)
    u = np.array([0.01, 0.02])
    me = O.meq(p, 1.0, u)
    f = Mi @ (me + d * np.eye(9)[1])
    mp = M @ O.collide_node(p, f, u)
    want = me.copy()
    want[1] += d * (1 - RATES[1])
    assert np.allclose(mp, want, atol=1e-15)
