"""Gaussian-hill validation sweeps on the batched GPU path (Sec. 3.1).

Every study of Sec. 3.1 is a set of independent periodic D2Q9 instances (one
per diffusion matrix, velocity, collision model, relaxation time or grid size),
so each runs as one ``Batch``: the instances advance together and each one's
phi is read back at its own time t_m (phi_max halved), where the errors of
Eq. 43 / 45 against the closed form of Eq. 41 are taken on the device.

  tables_1_2()        Tables 1-2: Er2, Er_inf of MRT-A/B1/B2/B3 for the three
                      diffusion matrices of Eq. 42, u = 0 and u = (0.05, 0.05)
  fig2_sweep(taus)    Fig. 2: Er2 against tau for the matrices of Eq. 44
  fig3_convergence()  Fig. 3: relative error (Eq. 45) against the grid size

Units: the paper's domain [-1, 1]^2 on 512 x 512 nodes gives dx = dt = 1/256,
so a physical D maps to the lattice D = D dt / dx^2 = 256 D, sigma0 = 0.05 to
12.8 nodes, and u keeps its value (dx = dt). The relaxation rates not fixed by
D are the set Sec. 3.1 gives: s1 = s2 = 1.1, s4 = s_xx, s6 = s_yy, s7 = s8 = 1.2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from .batch import Batch

DX = 1.0 / 256.0
# Eq. 42 (physical units, times 1e-4)
EQ42 = {
    "iso": np.array([[2.0, 0.0], [0.0, 2.0]]) * 1e-4,
    "diag": np.array([[1.0, 0.0], [0.0, 4.0]]) * 1e-4,
    "full": np.array([[1.0, 1.0], [1.0, 4.0]]) * 1e-4,
}
MODELS = ("A", "B1", "B2", "B3")
U_CONV = (0.05, 0.05)      # Table 2 / Fig. 2 convection-diffusion velocity


def lattice_D(D_phys, dx: float = DX) -> np.ndarray:
    """D dt / dx^2 with dt = dx."""
    return np.asarray(D_phys, dtype=np.float64) / dx


def eq44_D(kind: str, tau: float) -> np.ndarray:
    """Lattice D of Eq. 44: A^-1 = tau I, diag(tau, 4 tau - 1.5) or
    [[tau, tau - 1/2], [tau - 1/2, 4 tau - 1.5]], D = (I - A/2) A^-1 / 3."""
    if kind == "iso":
        Ai = np.array([[tau, 0.0], [0.0, tau]])
    elif kind == "diag":
        Ai = np.array([[tau, 0.0], [0.0, 4 * tau - 1.5]])
    elif kind == "full":
        Ai = np.array([[tau, tau - 0.5], [tau - 0.5, 4 * tau - 1.5]])
    else:
        raise ValueError(kind)
    return (Ai - 0.5 * np.eye(2)) / 3.0


def t_m(D, sigma0: float) -> float:
    """Time at which phi_max of Eq. 41 halves: det(sigma0^2 I + 2 t D) = 4 sigma0^4,
    i.e. 4 det(D) t^2 + 2 sigma0^2 tr(D) t - 3 sigma0^4 = 0 (positive root)."""
    D = np.asarray(D, dtype=np.float64)
    a, b, c = 4.0 * np.linalg.det(D), 2.0 * sigma0 ** 2 * np.trace(D), -3.0 * sigma0 ** 4
    if abs(a) < 1e-300:
        return -c / b
    return (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)


@dataclass
class Hill:
    """One periodic N x N instance: hill of width sigma0 (nodes) centred on node
    (N/2, N/2), lattice D, constant u, collision model, run for ``steps``."""

    N: int
    D: np.ndarray
    u: tuple = (0.0, 0.0)
    model: str = "A"
    sigma0: float = 12.8
    steps: int = 0
    tag: tuple = field(default_factory=tuple)

    def __post_init__(self):
        if self.steps <= 0:
            self.steps = int(round(t_m(self.D, self.sigma0)))

    def coords(self, device, dtype=torch.float64):
        j = torch.arange(self.N, device=device, dtype=dtype) - self.N // 2
        Y, X = torch.meshgrid(j, j, indexing="ij")
        return X, Y

    def phi0(self, device):
        X, Y = self.coords(device)
        return torch.exp(-(X * X + Y * Y) / (2 * self.sigma0 ** 2)).float()

    def exact(self, device, images: int = 1):
        """Eq. 41 at t = steps with total concentration 2 pi sigma0^2 (unit peak),
        summed over the periodic images within +-images boxes."""
        t = float(self.steps)
        st = self.sigma0 ** 2 * np.eye(2) + 2.0 * t * np.asarray(self.D, dtype=np.float64)
        si = np.linalg.inv(st)
        pref = self.sigma0 ** 2 / math.sqrt(np.linalg.det(st))
        X, Y = self.coords(device)
        out = torch.zeros_like(X)
        for a in range(-images, images + 1):
            for b in range(-images, images + 1):
                dx = X - self.u[0] * t - a * self.N
                dy = Y - self.u[1] * t - b * self.N
                out += torch.exp(-0.5 * (si[0, 0] * dx * dx + 2 * si[0, 1] * dx * dy + si[1, 1] * dy * dy))
        return pref * out


def errors(num: torch.Tensor, ana: torch.Tensor) -> dict:
    """Eq. 43 (Er2: root mean square, Er_inf: maximum) and Eq. 45 (relative L2)."""
    d = num.double() - ana
    return {"er2": float(torch.sqrt(torch.mean(d * d))), "er_inf": float(d.abs().max()),
            "er_rel": float(torch.linalg.norm(d) / torch.linalg.norm(ana))}


def run_hills(hills, device=None, mode="persistent", graph_steps=64):
    """Advance all instances in one Batch; return phi of each at its own steps."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    chans = []
    for h in hills:
        u = np.zeros((2, h.N), dtype=np.float32)
        u[0], u[1] = h.u
        chans.append({"nx": h.N, "ny": h.N, "bc": ("periodic", "periodic"), "D": h.D,
                      "u_row": u if any(h.u) else None, "model": h.model, "tie": True,
                      "s": [1.0, 1.1, 1.1, None, None, None, None, 1.2, 1.2]})
    b = Batch(chans, mode=mode, graph_steps=graph_steps, device=dev)
    try:
        b.set_phi([h.phi0(dev) for h in hills])
        out = [None] * len(hills)
        done = 0
        for stop in sorted({h.steps for h in hills}):
            b.run(stop - done, moments=False)
            done = stop
            phis = b.get_phi()
            for i, h in enumerate(hills):
                if h.steps == stop:
                    out[i] = phis[i].clone()
        torch.cuda.synchronize(dev)
    finally:
        b.close()
    return out


def _evaluate(hills, **kw):
    phis = run_hills(hills, **kw)
    return [errors(p, h.exact(p.device)) for p, h in zip(phis, hills)]


def tables_1_2(N: int = 512, models=MODELS, **kw) -> dict:
    """{(table, kind, model): errors} with table 1 (u = 0) and 2 (u = (0.05, 0.05))."""
    sig0 = 0.05 / DX * N / 512
    hills = []
    for table, u in ((1, (0.0, 0.0)), (2, U_CONV)):
        for kind, D in EQ42.items():
            for m in models:
                hills.append(Hill(N=N, D=lattice_D(D), u=u, model=m, sigma0=sig0, tag=(table, kind, m)))
    return {h.tag: e for h, e in zip(hills, _evaluate(hills, **kw))}


def fig2_sweep(taus, N: int = 512, kinds=("iso", "diag", "full"), velocities=((0.0, 0.0), U_CONV),
               models=MODELS, **kw) -> dict:
    """{(kind, u, model, tau): Er2} for the matrices of Eq. 44."""
    hills = []
    for kind in kinds:
        for u in velocities:
            for m in models:
                for tau in taus:
                    hills.append(Hill(N=N, D=eq44_D(kind, tau), u=tuple(u), model=m, sigma0=12.8,
                                      tag=(kind, tuple(u), m, float(tau))))
    return {h.tag: e["er2"] for h, e in zip(hills, _evaluate(hills, **kw))}


def fig3_convergence(Ns=(64, 128, 256, 512), kinds=("iso", "diag", "full"), model="A", **kw) -> dict:
    """{kind: (Ns, Er (Eq. 45), slope of ln Er against ln(1/N))}. dx = dt = 1/256
    as in Sec. 3.1, the domain side L = N dx / 2 and sigma0 = 0.05 L, so
    sigma0 = 0.025 N nodes and the lattice D is the same for every N."""
    hills = [Hill(N=n, D=lattice_D(EQ42[k]), model=model, sigma0=0.025 * n, tag=(k, n)) for k in kinds for n in Ns]
    res = {h.tag: e["er_rel"] for h, e in zip(hills, _evaluate(hills, **kw))}
    out = {}
    for k in kinds:
        ers = np.array([res[(k, n)] for n in Ns])
        slope = float(np.polyfit(np.log(1.0 / np.asarray(Ns, dtype=np.float64)), np.log(ers), 1)[0])
        out[k] = (list(Ns), ers.tolist(), slope)
    return out


def main():
    import argparse

    ap = argparse.ArgumentParser(description="Sec. 3.1 Gaussian-hill studies on the batched GPU path")
    ap.add_argument("--study", default="all", choices=["all", "tables", "fig2", "fig3"])
    ap.add_argument("--taus", default="0.55,0.6,0.7,0.8,1.0,1.2,1.5,2.0")
    args = ap.parse_args()
    if args.study in ("all", "tables"):
        res = tables_1_2()
        for table in (1, 2):
            print(f"Table {table}: Er2 / Er_inf at t_m, u = {(0, 0) if table == 1 else U_CONV}")
            for kind in EQ42:
                row = "  ".join(f"{m:>3} {res[(table, kind, m)]['er2']:.3e} {res[(table, kind, m)]['er_inf']:.3e}"
                                for m in MODELS)
                print(f"  {kind:5s} {row}")
    if args.study in ("all", "fig2"):
        taus = [float(t) for t in args.taus.split(",")]
        res = fig2_sweep(taus)
        for kind in ("iso", "diag", "full"):
            for u in ((0.0, 0.0), U_CONV):
                print(f"Fig. 2 {kind} u={u}: Er2 by tau {taus}")
                for m in MODELS:
                    print(f"  {m:>3} " + " ".join(f"{res[(kind, u, m, t)]:.3e}" for t in taus))
    if args.study in ("all", "fig3"):
        for kind, (Ns, ers, slope) in fig3_convergence().items():
            print(f"Fig. 3 {kind}: N {Ns} Er {['%.3e' % e for e in ers]} slope {slope:.3f}")


if __name__ == "__main__":
    main()
