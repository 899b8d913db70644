"""Sec. 3.1 studies on the batched GPU path (paper_1404_2363_gb300.validation):
periodic Gaussian-hill instances against the FP64 oracle, Tables 1-2 against
the printed values, the Fig. 2 relaxation-time sweep and the Fig. 3 order of
convergence."""
import math

import numpy as np
import pytest
import torch

from _common import rel_l2
from paper_1404_2363_gb300 import validation as V

pytestmark = pytest.mark.gpu

ORACLE_MODEL = {"A": 0, "B1": 1, "B2": 2, "B3": 3}


def test_hill_instances_match_oracle(O):
    """Every collision model with u = (0.05, 0.05), plus u = 0, on grids that leave
    ragged 32-column tiles, against the oracle after the same steps."""
    D = np.array([[0.03, 0.01], [0.01, 0.05]])
    hills = [V.Hill(N=48, D=D, u=V.U_CONV, model=m, sigma0=4.0, steps=90) for m in V.MODELS]
    hills.append(V.Hill(N=40, D=D, model="A", sigma0=4.0, steps=70))
    hills.append(V.Hill(N=40, D=D, model="B1", u=(0.08, -0.03), sigma0=4.0, steps=50))
    got = V.run_hills(hills)
    for h, g in zip(hills, got):
        p = O.Params(nx=h.N, ny=h.N, A=O.A_from_D(h.D), model=ORACLE_MODEL[h.model])
        u = np.zeros((2, h.N * h.N))
        u[0], u[1] = h.u
        want = O.run(p, h.phi0("cpu").double().numpy().reshape(-1), h.steps, u=u).reshape(h.N, h.N)
        assert rel_l2(g.cpu().numpy().astype(np.float64), want) <= 1e-5, h.model


def test_tables_1_2_on_gpu():
    """Tables 1-2 (512 x 512, t_m, Eq. 42 matrices): every Er2 and Er_inf within
    30 % of the printed value (the relaxation rates behind the tables are not
    printed; with the Sec. 3.1 set, MRT-B1 at u = 0 and MRT-B3 at u != 0 land
    within 4 %, MRT-A within 10 %, MRT-B1/B2 at u != 0 within 26 %), MRT-B2 equal
    to MRT-B3 at u = 0, and MRT-B3 well above the other models at u != 0."""
    import os

    res = V.tables_1_2()
    gold = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "gaussian_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, kind, *v = line.split()
        for j, m in enumerate(V.MODELS):
            gold[(int(t), kind, m)] = (float(v[2 * j]), float(v[2 * j + 1]))
    for key, want in gold.items():
        assert abs(res[key]["er2"] / want[0] - 1) < 0.30, (key, res[key], want)
        assert abs(res[key]["er_inf"] / want[1] - 1) < 0.30, (key, res[key], want)
    for kind in V.EQ42:
        assert res[(1, kind, "B2")]["er2"] == res[(1, kind, "B3")]["er2"]
        others = max(res[(2, kind, m)]["er2"] for m in ("A", "B1", "B2"))
        assert res[(2, kind, "B3")]["er2"] > 2.5 * others, kind


def test_fig3_second_order_on_gpu():
    """Fig. 3: the slope of ln Er against ln(1/N) is about 2 for the three matrices."""
    out = V.fig3_convergence(Ns=(64, 128, 256, 512, 1024))
    for kind, (Ns, ers, slope) in out.items():
        assert 1.85 < slope < 2.2, (kind, ers, slope)
        assert all(b < a for a, b in zip(ers, ers[1:])), (kind, ers)


def test_fig2_sweep_claims():
    """Fig. 2 (Eq. 44 matrices, tau from 0.55 to 2): at u = (0.05, 0.05) MRT-B3 has
    the largest Er2 at every tau, and MRT-A is below MRT-B1 and MRT-B2 at large tau;
    at u = 0 MRT-A is above the MRT-B models for most tau (the paper's "generally"),
    and MRT-B2 equals MRT-B3."""
    taus = [0.55, 0.6, 0.7, 0.8, 1.0, 1.2, 1.5, 2.0]
    res = V.fig2_sweep(taus)
    z, c = (0.0, 0.0), V.U_CONV
    for kind in ("iso", "diag", "full"):
        above = 0
        for t in taus:
            e = {m: res[(kind, c, m, t)] for m in V.MODELS}
            assert e["B3"] > max(e["A"], e["B1"], e["B2"]), (kind, t, e)
            if t >= 1.5:
                assert e["A"] < min(e["B1"], e["B2"]), (kind, t, e)
            e0 = {m: res[(kind, z, m, t)] for m in V.MODELS}
            assert e0["B2"] == e0["B3"]
            above += e0["A"] > max(e0["B1"], e0["B2"])
        assert above >= 6, (kind, above)
