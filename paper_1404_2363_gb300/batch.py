"""Torch-facing wrapper of the batched-channel C ABI (lbm_cde_batch_*).

Many independent D2Q9 channels (uneven size, own D, rates, walls and row
velocity profile) advance in one persistent launch or one launch per step,
replayed from a CUDA graph, with the Eq. 47 moments of every instance reduced
each step. ``alpha_L`` turns the moment series into the discrete Eq. 46
dispersion coefficient.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .solver import BC, MODELS, _TorchAllocator

MODES = {"auto": N.LBM_BATCH_AUTO, "persistent": N.LBM_BATCH_PERSISTENT, "per_step": N.LBM_BATCH_PER_STEP}


class Batch:
    def __init__(self, channels, mode="auto", tile_rows=0, graph_steps=64, barrier_timeout_cycles=2_000_000_000,
                 device=None, stream=None, torch_alloc=True):
        self.L = N.lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.n = len(channels)
        descs = (N.ChannelDesc * self.n)()
        self._keep = []
        self.shapes = []
        for d, ch in zip(descs, channels):
            d.nx, d.ny = int(ch["nx"]), int(ch["ny"])
            bc = ch.get("bc", ("noflux", "noflux"))
            d.bc_lo_y, d.bc_hi_y = BC[bc[0]], BC[bc[1]]
            D = np.asarray(ch["D"], dtype=np.float64).reshape(-1)
            for k in range(4):
                d.D[k] = float(D[k])
            s = ch.get("s")
            for k in range(15):
                d.s[k] = float("nan") if s is None or k >= len(s) or s[k] is None else float(s[k])
            d.tie_q_rates = 1 if ch.get("tie", True) else 0
            u = ch.get("u_row")
            if u is not None:
                u = torch.as_tensor(u, dtype=torch.float32).to(self.device).contiguous()
                self._keep.append(u)
                d.u_row_dev = u.data_ptr()
            d.x_ref0 = float(ch.get("x_ref0", 0.0))
            d.x_ref_velocity = float(ch.get("x_ref_velocity", 0.0))
            d.model = MODELS[ch.get("model", "A")]
            self.shapes.append((d.ny, d.nx))
        o = N.BatchOpts()
        self.L.lbm_cde_batch_opts_init(ctypes.byref(o))
        o.mode = MODES[mode]
        o.tile_rows = tile_rows
        o.graph_steps = graph_steps
        o.barrier_timeout_cycles = int(barrier_timeout_cycles)
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(self.device, self.stream)
            o.alloc, o.free_ = self._alloc.alloc_fn, self._alloc.free_fn
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        st = self.L.lbm_cde_batch_create(descs, self.n, ctypes.byref(o), ctypes.byref(h))
        if st != N.LBM_OK:
            raise N.LbmError(st, "lbm_cde_batch_create", self.L.lbm_cde_batch_last_error(None).decode())
        self.h = h
        v = ctypes.c_int64()
        self._ck(self.L.lbm_cde_batch_cells(self.h, ctypes.byref(v)), "lbm_cde_batch_cells")
        self.ncat = v.value
        self.offsets = np.cumsum([0] + [a * b for a, b in self.shapes])

    def _ck(self, st, what):
        if st != N.LBM_OK:
            raise N.LbmError(st, what, self.L.lbm_cde_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_cde_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def concat(self, fields):
        return torch.cat([torch.as_tensor(f, dtype=torch.float32).reshape(-1) for f in fields]).to(self.device)

    def split(self, flat):
        flat = flat.reshape(-1)
        return [flat[self.offsets[i]:self.offsets[i + 1]].reshape(self.shapes[i]) for i in range(self.n)]

    def set_phi(self, fields):
        phi = self.concat(fields).contiguous()
        self._phi0 = phi
        self._ck(self.L.lbm_cde_batch_set_phi(self.h, phi.data_ptr()), "lbm_cde_batch_set_phi")

    def get_phi(self):
        out = torch.empty(self.ncat, device=self.device, dtype=torch.float32)
        self._ck(self.L.lbm_cde_batch_get_phi(self.h, out.data_ptr()), "lbm_cde_batch_get_phi")
        return self.split(out)

    def run(self, nsteps, moments=True):
        m = np.zeros((nsteps, self.n, 3)) if moments else None
        self._ck(self.L.lbm_cde_batch_run(self.h, int(nsteps), m.ctypes.data_as(N._DP) if m is not None else None),
                 "lbm_cde_batch_run")
        return m

    def autotune(self, steps=64):
        mode, tile = ctypes.c_int32(), ctypes.c_int32()
        self._ck(self.L.lbm_cde_batch_autotune(self.h, int(steps), ctypes.byref(mode), ctypes.byref(tile)),
                 "lbm_cde_batch_autotune")
        return {1: "persistent", 2: "per_step"}[mode.value], tile.value

    def config(self, mode, tile_rows):
        self._ck(self.L.lbm_cde_batch_config(self.h, MODES[mode], int(tile_rows)), "lbm_cde_batch_config")


def sigma2(moments):
    """Eq. 47 from the moment sums."""
    m0, m1, m2 = moments[..., 0], moments[..., 1], moments[..., 2]
    return m2 / m0 - (m1 / m0) ** 2


def alpha_L(moments, window=1):
    """Discrete Eq. 46 over `window` steps: (sigma^2_{n+w} - sigma^2_n) / (2 w)."""
    s2 = sigma2(moments)
    return (s2[window:] - s2[:-window]) / (2.0 * window)


def poiseuille_row(ny, U):
    y = np.arange(ny, dtype=np.float64)
    W = ny - 1
    u = np.zeros((2, ny), dtype=np.float32)
    u[0] = (4.0 * U * y * (W - y) / (W * W)).astype(np.float32)
    return u


def mean_velocity(u_row):
    """Trapezoid mean of u_x over the nodes (walls on the nodes)."""
    w = np.ones(u_row.shape[1])
    w[0] = w[-1] = 0.5
    return float((w * u_row[0]).sum() / w.sum())
