"""Writes taylor_aris_mrt_a_oracle.txt beside this script: the oracle's MRT-A
relative error Er x 100 of the converged longitudinal dispersion coefficient
(Sec. 3.2, Eq. 46-49) for the channel of Tables 3-5 with the printed rates,
signed (numeric minus analytic), at every (tau, Pe) of the tables; and prints
how those errors move when one reading of the set-up is changed at a time.

Calls only the oracle (oracle/), as the recorded values of the test suite must.

    python tests/golden/make_taylor_aris_mrt_a.py [--study]
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

OUT = os.path.join(HERE, "taylor_aris_mrt_a_oracle.txt")
TABLES = os.path.join(HERE, "taylor_aris_tables.txt")


def table_rows():
    rows = []
    for line in open(TABLES):
        if line.startswith("#") or not line.strip():
            continue
        t, tau, Pe, *er = line.split()
        rows.append((int(t), float(tau), float(Pe), [float(v) for v in er]))
    return rows


def signed_er(tau, Pe, model=O.MRT_A, s1=1.1, s2=1.1, s7=1.2, s8=1.2, trapezoid=True, W=32):
    """Sec. 3.2 channel: W lattices between wall nodes (Neumann rule), Poiseuille
    u_x at the nodes, D = alpha I with alpha = (tau - 1/2)/3, Pe = 2 U W / (3 alpha);
    the x-moments of a unit pulse by the oracle's exact channel recursion."""
    ny = W + 1
    alpha = (tau - 0.5) / 3.0
    U = 3.0 * alpha * Pe / (2.0 * W)
    y = np.arange(ny, dtype=float)
    ux = 4.0 * U * y * (W - y) / W ** 2
    s = np.array([1.0, s1, s2, 0.0, 1 / tau, 0.0, 1 / tau, s7, s8])
    p = O.Params(q=9, model=model, nx=1, ny=ny, bc_lo=O.NOFLUX_NODE, bc_hi=O.NOFLUX_NODE,
                 A=np.eye(2) / tau, s=s, tie=False)
    _, _, Mi, _ = O.tables(p)
    F0 = np.zeros((3, 9, ny))
    for yy in range(ny):
        F0[0, :, yy] = Mi @ O.meq(p, 1.0, [ux[yy], 0.0])
    wy = np.ones(ny)
    if trapezoid:
        wy[0] = wy[-1] = 0.5
    nsteps = 30000 if tau >= 1.0 else 200000
    a = O.alpha_series(O.channel_moments(p, ux, F0, wy, nsteps))
    an = O.taylor_aris_analytic(alpha, Pe)
    return (a[-1] - an) / an * 100.0


READINGS = [
    ("printed rates (s1 = s2 = 1.1, s7 = s8 = 1.2), trapezoid cross-section mean", {}),
    ("s1 = 1.0", {"s1": 1.0}),
    ("s1 = 1.2", {"s1": 1.2}),
    ("s2 = 1.0", {"s2": 1.0}),
    ("s2 = 1.2", {"s2": 1.2}),
    ("s7 = s8 = 1.0", {"s7": 1.0, "s8": 1.0}),
    ("s7 = s8 = 1.5", {"s7": 1.5, "s8": 1.5}),
    ("plain cross-section mean (weight 1 on the wall nodes)", {"trapezoid": False}),
]


def main():
    rows = table_rows()
    with open(OUT, "w") as fh:
        fh.write("# Oracle MRT-A Er x 100 (signed: numeric minus analytic) for the Sec. 3.2 channel with the\n")
        fh.write("# printed rates, written by make_taylor_aris_mrt_a.py (oracle only).\n")
        fh.write("# columns: table tau Pe oracle_signed_Er_x100 printed_MRT-A |oracle|/printed\n")
        for t, tau, Pe, er in rows:
            v = signed_er(tau, Pe)
            fh.write(f"{t} {tau} {Pe:g} {v:+.6f} {er[0]:.6f} {abs(v) / er[0]:.4f}\n")
    print(open(OUT).read())
    if "--study" in sys.argv:
        cases = [(2.0, 4.0), (1.0, 8.0), (0.55, 32.0)]
        printed = {(tau, Pe): er[0] for _, tau, Pe, er in rows}
        print("| reading | " + " | ".join(f"tau = {t}, Pe = {p:g}" for t, p in cases) + " |")
        print("|---|" + "---|" * len(cases))
        for name, kw in READINGS:
            vals = [signed_er(t, p, **kw) for t, p in cases]
            print(f"| {name} | " + " | ".join(f"{v:+.5f} ({abs(v) / printed[c]:.3f})"
                                             for v, c in zip(vals, cases)) + " |")


if __name__ == "__main__":
    main()
