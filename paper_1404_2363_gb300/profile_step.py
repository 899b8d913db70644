"""Runs a few steps of one solver configuration, for profilers.

  python -m paper_1404_2363_gb300.profile_step --lattice 9 --storage f32 --n 2048 --steps 4

The grid is n x n (D2Q9) or n^3 (D3Q15), periodic, with a random velocity
field and a Gaussian hill; the state is larger than L2 for n >= 2048 (2D)
and n >= 128 (3D), so DRAM counters reflect the streaming traffic.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import workloads as W
from .solver import Solver


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", type=int, default=9)
    ap.add_argument("--storage", default="f32")
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--ukind", default="field", choices=["none", "field"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--vec", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0, help="run N Taylor-Aris channels (per-step mode) instead")
    ap.add_argument("--tile", type=int, default=16, help="rows per batch warp tile")
    ap.add_argument("--mode", default="per_step", choices=["per_step", "persistent"])
    ap.add_argument("--adjoint", action="store_true", help="forward_ckpt + backward (dL/dD, dL/da)")
    args = ap.parse_args()
    if args.batch:
        return run_batch(args)
    n = args.n
    if args.lattice == 9:
        shape, dim = (n, n), 2
        D = W.D_eq44_full(1.0)
    else:
        shape, dim = (n, n, n), 3
        D = np.diag([0.02, 0.03, 0.04])
    s = Solver(lattice=args.lattice, nx=n, ny=n, nz=1 if args.lattice == 9 else n, storage=args.storage)
    if args.block:
        s.set_launch(args.block, args.vec or 1)
    s.set_D(D)
    g = np.random.default_rng(0)
    if args.ukind == "field":
        a = torch.from_numpy(g.uniform(-0.05, 0.05, (dim,) + shape).astype(np.float32)).cuda()
        s.set_velocity(a)
    phi0 = torch.from_numpy((0.5 + g.random(shape)).astype(np.float32)).cuda()
    if args.adjoint:
        s.forward_ckpt(phi0, args.steps)
        _, dD, _, _ = s.backward(torch.ones(shape, device="cuda"), want_da=args.ukind == "field")
        s.close()
        print(f"ok adjoint n={n} steps={args.steps} dL/dD[0,0]={dD[0, 0]:.6e}")
        return
    s.set_phi(phi0)
    s.step(args.steps)
    m = s.sum_phi()
    s.close()
    print(f"ok lattice={args.lattice} storage={args.storage} n={n} steps={args.steps} sum_phi={m:.6e}")


def run_batch(args):
    from .batch import Batch, mean_velocity, poiseuille_row

    chans = W.taylor_aris_batch(args.batch)
    descs, phis = [], []
    for c in chans:
        u = poiseuille_row(c.ny, c.U)
        descs.append({"nx": c.nx, "ny": c.ny, "D": np.eye(2) * c.alpha, "u_row": u, "tie": False,
                      "s": [1.0, 1.1, 1.1, None, 1 / c.tau, None, 1 / c.tau, 1.2, 1.2],
                      "x_ref0": 0.2 * c.nx, "x_ref_velocity": mean_velocity(u)})
        phis.append(c.phi0().astype(np.float32))
    b = Batch(descs, mode=args.mode, tile_rows=args.tile, graph_steps=1)
    b.set_phi(phis)
    m = b.run(args.steps)
    b.close()
    print(f"ok batch={args.batch} cells={b.ncat} steps={args.steps} m0={m[-1, 0, 0]:.6e}")


if __name__ == "__main__":
    main()
