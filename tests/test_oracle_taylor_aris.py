"""Taylor-Aris dispersion pins (Sec. 3.2, Eq. 46-49, Tables 3-5).

The oracle's exact x-moment recursion for a channel (``channel_moments``) is
first checked against the oracle's full 2D step on a short channel; then its
converged dispersion coefficient is compared with the paper's printed errors
(tests/golden/taylor_aris_tables.txt).

Tolerance: the paper stops at the first n with (a_{n+100} - a_n)/a_n <= 1e-6
(Eq. 49), which leaves a_n within a few 1e-6 of its limit; the Er x 100 values
therefore carry an uncertainty of a few 1e-4 in absolute terms. We compare the
converged limit with max(1 % relative, 5e-4 absolute).

MRT-B1, B2 and B3 reproduce every checked entry within that tolerance, which
pins M, the equilibria of Eq. 37-39, the unmodified S, the wall rule, the
streaming and the estimator. MRT-A (modified S, Eq. 31) reproduces the printed
MRT-A column's dependence on Pe at each tau (the ratio of our error to the
printed one is the same for all four Pe of a table, to 0.2 %; a weak pin, since
any error proportional to the Taylor part Pe^2 / 210 of alpha_L has that
shape), but not its level: the ratio is 1.314 at tau = 2, 2.058 at tau = 1 and 0.961 at tau = 0.55.
No single change of reading moves all three levels onto the printed ones
(tests/golden/make_taylor_aris_mrt_a.py --study varies the free rates s1, s2,
s7 = s8 and the cross-section weighting one at a time); the level is pinned
instead by the exact deviation-free variance growth of the modified S
(tests/test_oracle_step.py) and the hand-computed collisions
(tests/test_oracle_collision.py), and here by the recorded oracle values
(tests/golden/taylor_aris_mrt_a_oracle.txt, written by that script).
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "taylor_aris_tables.txt")


def load_tables():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t, tau, Pe, *er = line.split()
        rows.append((int(t), float(tau), float(Pe), [float(v) for v in er]))
    return rows


def channel(O, tau, Pe, model, W=32):
    ny = W + 1
    alpha = (tau - 0.5) / 3.0
    U = 3.0 * alpha * Pe / (2.0 * W)          # Pe = 2 U W / (3 alpha)
    y = np.arange(ny, dtype=float)
    ux = 4.0 * U * y * (W - y) / W ** 2
    s = np.array([1.0, 1.1, 1.1, 0.0, 1 / tau, 0.0, 1 / tau, 1.2, 1.2])
    p = O.Params(q=9, model=model, nx=1, ny=ny, bc_lo=O.NOFLUX_NODE, bc_hi=O.NOFLUX_NODE,
                 A=np.eye(2) / tau, s=s, tie=False)
    return p, ux, alpha


def converged_er(O, tau, Pe, model, nsteps, signed=False):
    p, ux, alpha = channel(O, tau, Pe, model)
    ny = p.ny
    _, M, Mi, _ = O.tables(p)
    F0 = np.zeros((3, 9, ny))
    for yy in range(ny):
        F0[0, :, yy] = Mi @ O.meq(p, 1.0, [ux[yy], 0.0])   # pulse of unit mass at x = 0
    wy = np.ones(ny)
    wy[0] = wy[-1] = 0.5
    a = O.alpha_series(O.channel_moments(p, ux, F0, wy, nsteps))
    an = O.taylor_aris_analytic(alpha, Pe)
    # the limit has been reached: the last 1000 steps agree to 1e-7 (the
    # residual is FP64 cancellation in <x^2> - <x>^2, far below the tolerance)
    assert abs(a[-1] - a[-1000]) / a[-1] < 1e-7
    return ((a[-1] - an) if signed else abs(a[-1] - an)) / an * 100.0


def test_moment_recursion_equals_full_2d_oracle(O):
    """Exact identity: x-moments from the full 2D push-form step on a periodic
    channel equal the recursion while the pulse stays clear of the seam."""
    tau, Pe = 1.2, 20.0
    for model in (O.MRT_A, O.MRT_B1):
        p1, ux, _ = channel(O, tau, Pe, model)
        nx, ny = 400, p1.ny
        p2 = O.Params(q=9, model=model, nx=nx, ny=ny, bc_lo=O.NOFLUX_NODE, bc_hi=O.NOFLUX_NODE,
                      A=p1.A, s=p1.s, tie=False)
        phi0 = np.zeros((ny, nx))
        phi0[:, 150:156] = 1.0
        u = np.zeros((2, ny, nx))
        u[0] = ux[:, None]
        nsteps = 100
        f = O.init_eq(p2, phi0, u.reshape(2, -1))
        wy = np.ones(ny)
        wy[0] = wy[-1] = 0.5
        x = np.arange(nx, dtype=float)
        full = []
        for t in range(nsteps + 1):
            phi = O.phi_of(p2, f).reshape(ny, nx)
            pbar = (wy[:, None] * phi).sum(axis=0)
            full.append([pbar.sum(), (x * pbar).sum(), (x * x * pbar).sum()])
            if t < nsteps:
                f = O.step(p2, f, u.reshape(2, -1))
        full = np.array(full)
        _, _, Mi, _ = O.tables(p1)
        F0 = np.zeros((3, 9, ny))
        for yy in range(ny):
            fe = Mi @ O.meq(p1, 1.0, [ux[yy], 0.0])
            for k in range(3):
                F0[k, :, yy] = fe * (x ** k * phi0[yy]).sum()
        rec = O.channel_moments(p1, ux, F0, wy, nsteps)
        assert np.allclose(rec, full, rtol=1e-12, atol=1e-12)


def test_analytic_alpha_L():
    import oracle as O

    assert O.taylor_aris_analytic(0.5, 0.0) == 0.5
    assert abs(O.taylor_aris_analytic(0.2, math.sqrt(210.0)) - 0.4) < 1e-15


CASES = [(2.0, 2), (2.0, 16), (1.0, 4), (1.0, 32), (0.55, 16), (0.55, 128)]


@pytest.mark.parametrize("tau,Pe", CASES)
def test_b_models_reproduce_tables_3_to_5(O, tau, Pe):
    table = {(r[1], r[2]): r[3] for r in load_tables()}
    want = table[(tau, float(Pe))]
    nsteps = 30000 if tau >= 1.0 else 200000
    ours = [converged_er(O, tau, Pe, m, nsteps) for m in (O.MRT_A, O.MRT_B1, O.MRT_B2, O.MRT_B3)]
    for k in (1, 2, 3):
        assert abs(ours[k] - want[k]) <= max(0.01 * want[k], 5e-4), (k, ours[k], want[k])
    # MRT-A: the paper's ordering against the B models holds (Sec. 3.2)
    if tau >= 1.0:
        assert ours[0] < min(ours[1:])
    else:
        assert ours[0] < ours[3] < ours[1] < ours[2]


def recorded_mrt_a():
    path = os.path.join(os.path.dirname(__file__), "golden", "taylor_aris_mrt_a_oracle.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t, tau, Pe, signed, printed, ratio = line.split()
        out[(float(tau), float(Pe))] = (float(signed), float(printed))
    return out


@pytest.mark.parametrize("tau", [2.0, 1.0, 0.55])
def test_mrt_a_pe_dependence_matches_the_printed_column(O, tau):
    """At fixed tau the oracle's MRT-A error is the printed MRT-A error times one
    factor for every Pe of the table (0.5 %): the velocity dependence of the
    modified model matches Tables 3-5; the factor itself is the recorded
    discrepancy of the level, checked against the recorded oracle values (1 %)."""
    table = {(r[1], r[2]): r[3] for r in load_tables()}
    rec = recorded_mrt_a()
    nsteps = 30000 if tau >= 1.0 else 200000
    ratios = []
    for (t, Pe), er in sorted(table.items()):
        if t != tau:
            continue
        signed = converged_er(O, tau, Pe, O.MRT_A, nsteps, signed=True)
        want_signed, printed = rec[(tau, Pe)]
        assert abs(signed - want_signed) <= 0.01 * abs(want_signed), (tau, Pe, signed, want_signed)
        ratios.append(abs(signed) / er[0])
    assert len(ratios) == 4
    assert max(ratios) / min(ratios) - 1.0 < 5e-3, ratios


def test_error_ratio_nearly_independent_of_pe(O):
    """Sec. 3.2: at fixed tau the ratio Er_A : Er_B* barely changes with Pe."""
    r = []
    for Pe in (2, 8):
        ea = converged_er(O, 2.0, Pe, O.MRT_A, 30000)
        eb = converged_er(O, 2.0, Pe, O.MRT_B1, 30000)
        r.append(eb / ea)
    assert abs(r[1] - r[0]) / r[0] < 0.01
