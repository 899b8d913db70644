"""Helpers shared by the GPU parity tests: one case description drives both
the CUDA path (through the C ABI) and the FP64 oracle, on the same seeded
float32 inputs."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from paper_1404_2363_gb300 import workloads as W

BC_ORACLE = {"periodic": 0, "noflux": 1, "bounceback": 2, "dirichlet": 3}


@dataclass
class Case:
    lattice: int = 9
    nx: int = 300
    ny: int = 37
    nz: int = 1
    storage: str = "f32"
    bc: tuple = ("periodic", "periodic")
    phi_w: tuple = (0.0, 0.0)
    ukind: str = "field"          # none | field | row
    sched: bool = True
    steps: int = 200
    D: np.ndarray = field(default_factory=lambda: W.D_ANISO.copy())
    umax: float = 0.05
    seed: int = 0
    model: str = "A"
    bg: bool = True               # False: the hill alone, no positive background
    bc_x: tuple = ("periodic", "periodic")
    bc_z: tuple = ("periodic", "periodic")

    @property
    def dim(self):
        return 2 if self.lattice == 9 else 3

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.lattice == 15 else (self.ny, self.nx)

    def inputs(self):
        g = np.random.default_rng(1234 + self.seed)
        if self.lattice == 9:
            phi0 = W.gaussian_phi0(self.nx, self.ny, max(self.nx, self.ny) / 8.0)
            if self.bg:
                phi0 = phi0 + 0.2 + 0.1 * g.random(self.shape)
        elif self.bg:
            phi0 = 0.5 + g.random(self.shape)
        else:
            z, y, x = np.meshgrid(np.arange(self.nz) - self.nz / 2, np.arange(self.ny) - self.ny / 2,
                                  np.arange(self.nx) - self.nx / 2, indexing="ij")
            r = max(self.nx, self.ny, self.nz) / 6.0
            phi0 = np.exp(-(x * x + y * y + z * z) / (2 * r * r))
        phi0 = phi0.astype(np.float32)
        a = None
        if self.ukind == "field":
            a = g.uniform(-self.umax, self.umax, (self.dim,) + self.shape).astype(np.float32)
            if self.bc[0] != "periodic":
                a[1] *= 0.2      # keep wall-normal flow small near walls
            if self.bc_x[0] != "periodic":
                a[0] *= 0.2
            if self.bc_z[0] != "periodic":
                a[2] *= 0.2
        elif self.ukind == "row":
            y = np.arange(self.ny, dtype=np.float64)
            W_ = self.ny - 1
            a = np.zeros((self.dim, self.ny), dtype=np.float32)
            a[0] = (4 * self.umax * y * (W_ - y) / W_ ** 2).astype(np.float32)
        sched = None
        if self.sched and a is not None:
            t = np.arange(64)
            sched = np.stack([np.cos(2 * np.pi * t / 64 + k) for k in range(self.dim)], axis=1).astype(np.float32)
        return phi0, a, sched

    def u_of_t(self, a, sched):
        """Velocity field at step t in FP64 from the same float32 inputs."""
        if a is None:
            return None
        n = int(np.prod(self.shape))
        if self.ukind == "row":
            idx = (slice(None), None) if self.lattice == 9 else (None, slice(None), None)
            full = np.stack([np.broadcast_to(a[d].astype(np.float64)[idx], self.shape)
                             for d in range(self.dim)])
            base = full.reshape(self.dim, n)
        else:
            base = a.astype(np.float64).reshape(self.dim, n)
        if sched is None:
            return lambda t: base
        s = sched.astype(np.float64)
        return lambda t: base * s[t % len(s)][:, None]


def oracle_params(O, case: Case):
    kw = dict(nx=case.nx, ny=case.ny, nz=case.nz,
              bc_lo=BC_ORACLE[case.bc[0]], bc_hi=BC_ORACLE[case.bc[1]],
              phi_w_lo=case.phi_w[0], phi_w_hi=case.phi_w[1],
              bcx_lo=BC_ORACLE[case.bc_x[0]], bcx_hi=BC_ORACLE[case.bc_x[1]],
              bcz_lo=BC_ORACLE[case.bc_z[0]], bcz_hi=BC_ORACLE[case.bc_z[1]])
    if case.lattice == 9:
        model = {"A": O.MRT_A, "B1": O.MRT_B1, "B2": O.MRT_B2, "B3": O.MRT_B3}[case.model]
        return O.Params(A=O.A_from_D(case.D), model=model, **kw)
    return O.default_params_3d(A=O.A_from_D(case.D, q=15, alpha1=-1.2, alpha2=192.0), **kw)


def run_oracle(O, case: Case, phi0, a, sched, steps=None):
    p = oracle_params(O, case)
    steps = case.steps if steps is None else steps
    uf = case.u_of_t(a, sched)
    phi = O.run(p, phi0.astype(np.float64).reshape(-1), steps, u_of_t=uf) if uf is not None else \
        O.run(p, phi0.astype(np.float64).reshape(-1), steps)
    return phi.reshape(case.shape)


def run_gpu(case: Case, phi0, a, sched, steps=None, solver_kw=None):
    import torch

    from paper_1404_2363_gb300.solver import Solver

    steps = case.steps if steps is None else steps
    s = Solver(lattice=case.lattice, nx=case.nx, ny=case.ny, nz=case.nz, storage=case.storage,
               bc=case.bc, phi_w=case.phi_w, model=case.model, bc_x=case.bc_x, bc_z=case.bc_z,
               **(solver_kw or {}))
    s.set_D(case.D)
    if a is not None:
        s.set_velocity(torch.from_numpy(a).cuda(), None if sched is None else torch.from_numpy(sched).cuda(),
                       kind="row" if case.ukind == "row" else "field")
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(steps)
    out = s.get_phi().cpu().numpy().astype(np.float64)
    return out, s


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rel_max(a, b):
    """max |a - b| over max |b|: a per-element bound that a background cannot dilute."""
    return float(np.abs(a - b).max() / np.abs(b).max())


def assert_parity(got, want, tol, what=""):
    """Relative L2 and per-element (max |error| over max |phi|) bounds, both at tol."""
    e2, em = rel_l2(got, want), rel_max(got, want)
    assert e2 <= tol and em <= tol, (what, e2, em, tol)
    return e2, em
