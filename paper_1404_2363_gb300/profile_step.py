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
    args = ap.parse_args()
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
    s.set_phi(phi0)
    s.step(args.steps)
    m = s.sum_phi()
    s.close()
    print(f"ok lattice={args.lattice} storage={args.storage} n={n} steps={args.steps} sum_phi={m:.6e}")


if __name__ == "__main__":
    main()
