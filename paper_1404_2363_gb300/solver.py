"""Thin torch-facing wrapper over the C ABI (device memory and streams from torch).

``Solver`` marshals tensors into the ``lbm_cde_*`` calls; every step of the
method runs in the CUDA kernels of liblbm_cde.so.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native as N

STORAGE = {"f32": N.LBM_STORE_F32, "f16": N.LBM_STORE_F16_NEQ, "bf16": N.LBM_STORE_BF16_NEQ}
MODELS = {"A": N.LBM_MRT_A, "B1": N.LBM_MRT_B1, "B2": N.LBM_MRT_B2, "B3": N.LBM_MRT_B3}
BC = {"periodic": N.LBM_BC_PERIODIC, "noflux": N.LBM_BC_NOFLUX_NODE,
      "bounceback": N.LBM_BC_BOUNCEBACK, "dirichlet": N.LBM_BC_DIRICHLET}


class _TorchAllocator:
    """Device allocations of the handle go through torch's caching allocator."""

    def __init__(self, device: torch.device, stream: torch.cuda.Stream):
        self.device = device
        self.stream = stream
        self.alloc_fn = N.ALLOC_FN(self._alloc)
        self.free_fn = N.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), self.device.index, self.stream)
        except Exception:  # noqa: BLE001 - reported as LBM_E_OOM by the library
            return None

    def _free(self, ptr, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)


class Solver:
    """One lattice Boltzmann solver instance on one GPU.

    Parameters mirror ``lbm_cde_desc``: lattice 9 (D2Q9) or 15 (D3Q15), grid
    (nx, ny, nz), storage 'f32' | 'f16' | 'bf16', wall kinds for the y faces
    (``bc``) and for the x and z faces (``bc_x``, ``bc_z``: periodic, noflux or
    bounceback),
    Dirichlet values, optional alpha1/alpha2 and diagonal rates ``s`` (None
    entries keep the defaults).
    """

    def __init__(self, lattice=9, nx=64, ny=64, nz=1, storage="f32", bc=("periodic", "periodic"),
                 phi_w=(0.0, 0.0), alpha=None, s=None, tie=True, device=None, stream=None,
                 torch_alloc=True, model="A", bc_x=("periodic", "periodic"), bc_z=("periodic", "periodic")):
        self.L = N.lib()
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.dim = 2 if lattice == 9 else 3
        self.lattice = lattice
        self.shape = (nz, ny, nx) if lattice == 15 else (ny, nx)
        self.ncell = nx * ny * nz
        d = N.LbmDesc()
        N.check(self.L.lbm_cde_desc_init(ctypes.byref(d), lattice, nx, ny, nz), "desc_init")
        d.storage = STORAGE[storage]
        d.bc_lo_y, d.bc_hi_y = BC[bc[0]], BC[bc[1]]
        d.bc_lo_x, d.bc_hi_x = BC[bc_x[0]], BC[bc_x[1]]
        d.bc_lo_z, d.bc_hi_z = BC[bc_z[0]], BC[bc_z[1]]
        d.phi_w_lo_y, d.phi_w_hi_y = float(phi_w[0]), float(phi_w[1])
        if alpha is not None:
            d.alpha1, d.alpha2 = float(alpha[0]), float(alpha[1])
        if s is not None:
            for k, v in enumerate(s):
                if v is not None and not (isinstance(v, float) and math.isnan(v)):
                    d.s[k] = float(v)
        d.tie_q_rates = 1 if tie else 0
        d.model = MODELS[model]
        self._alloc = None
        if torch_alloc:
            self._alloc = _TorchAllocator(self.device, self.stream)
            d.alloc = self._alloc.alloc_fn
            d.free_ = self._alloc.free_fn
        d.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.desc = d
        h = ctypes.c_void_p()
        N.check(self.L.lbm_cde_create(ctypes.byref(d), ctypes.byref(h)), "lbm_cde_create")
        self.h = h
        self._keep = []

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_cde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _ck(self, st, what):
        N.check(st, what, self.h)

    # -- parameters -------------------------------------------------------
    def set_D(self, D):
        D = np.ascontiguousarray(np.asarray(D, dtype=np.float64).reshape(self.dim, self.dim))
        self._ck(self.L.lbm_cde_set_D(self.h, D.ctypes.data_as(N._DP)), "lbm_cde_set_D")

    def rates(self):
        A = np.zeros(self.dim * self.dim)
        s = np.zeros(15)
        self._ck(self.L.lbm_cde_get_rates(self.h, A.ctypes.data_as(N._DP), s.ctypes.data_as(N._DP)),
                 "lbm_cde_get_rates")
        return A.reshape(self.dim, self.dim), s

    def set_velocity(self, a=None, sched=None, kind="field"):
        """a: float32 tensor (dim, *grid) for kind='field' or (dim, ny) for
        kind='row'; sched: float32 (len, dim) multipliers s(t), or None."""
        if a is None:
            self._keep = []
            self._ck(self.L.lbm_cde_set_velocity(self.h, N.LBM_U_NONE, None, None, 0),
                     "lbm_cde_set_velocity")
            return
        a = a.to(self.device, torch.float32).contiguous()
        kind = {"field": N.LBM_U_FIELD, "row": N.LBM_U_ROW_PROFILE}[kind]
        sp, sl = None, 0
        if sched is not None:
            sched = sched.to(self.device, torch.float32).contiguous()
            sp, sl = sched.data_ptr(), sched.shape[0]
        self._keep = [a, sched]
        self._ck(self.L.lbm_cde_set_velocity(self.h, kind, a.data_ptr(), sp, sl), "lbm_cde_set_velocity")

    # -- state ------------------------------------------------------------
    def set_phi(self, phi):
        phi = phi.to(self.device, torch.float32).contiguous()
        self._phi0 = phi
        self._ck(self.L.lbm_cde_set_phi(self.h, phi.data_ptr()), "lbm_cde_set_phi")

    def set_launch(self, block=256, vec=1):
        self._ck(self.L.lbm_cde_set_launch(self.h, int(block), int(vec)), "lbm_cde_set_launch")

    def set_wait_limit(self, cycles):
        """Bound (SM clock cycles) on each device wait of the TMA-staged kernel."""
        self._ck(self.L.lbm_cde_set_wait_limit(self.h, int(cycles)), "lbm_cde_set_wait_limit")

    def set_zwalk(self, planes):
        """Planes per CTA of the D3Q15 z-walk kernel (0: chosen by the launcher)."""
        self._ck(self.L.lbm_cde_set_zwalk(self.h, int(planes)), "lbm_cde_set_zwalk")

    def autotune(self, steps=20):
        b, v = ctypes.c_int32(), ctypes.c_int32()
        self._ck(self.L.lbm_cde_autotune(self.h, int(steps), ctypes.byref(b), ctypes.byref(v)), "lbm_cde_autotune")
        return b.value, v.value

    def step(self, n=1):
        self._ck(self.L.lbm_cde_step(self.h, int(n)), "lbm_cde_step")

    @property
    def t(self):
        v = ctypes.c_int64()
        self._ck(self.L.lbm_cde_get_time(self.h, ctypes.byref(v)), "lbm_cde_get_time")
        return v.value

    def get_phi(self, out=None):
        if out is None:
            out = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        self._ck(self.L.lbm_cde_get_phi(self.h, out.data_ptr()), "lbm_cde_get_phi")
        return out

    def sum_phi(self):
        v = ctypes.c_double()
        self._ck(self.L.lbm_cde_sum_phi(self.h, ctypes.byref(v)), "lbm_cde_sum_phi")
        return v.value

    def sync(self):
        """Waits for the stream; reports a latched device status (LBM_E_TIMEOUT)."""
        self._ck(self.L.lbm_cde_sync(self.h), "lbm_cde_sync")

    def state_bytes(self):
        v = ctypes.c_size_t()
        self._ck(self.L.lbm_cde_state_bytes(self.h, ctypes.byref(v)), "lbm_cde_state_bytes")
        return v.value

    def get_state(self, out=None):
        if out is None:
            out = torch.empty(self.state_bytes(), device=self.device, dtype=torch.uint8)
        t = ctypes.c_int64()
        self._ck(self.L.lbm_cde_get_state(self.h, out.data_ptr(), ctypes.byref(t)), "lbm_cde_get_state")
        return out, t.value

    def set_state(self, buf, t):
        self._ck(self.L.lbm_cde_set_state(self.h, buf.data_ptr(), int(t)), "lbm_cde_set_state")

    # -- differentiation -------------------------------------------------
    def forward_ckpt(self, phi0, nsteps, every=0, out=None):
        """phi after nsteps from f^eq(phi0, u(0)), keeping checkpoints for backward()."""
        phi0 = phi0.to(self.device, torch.float32).contiguous()
        self._phi0 = phi0
        if out is None:
            out = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        self._ck(self.L.lbm_cde_forward_ckpt(self.h, phi0.data_ptr(), int(nsteps), int(every), out.data_ptr()),
                 "lbm_cde_forward_ckpt")
        return out

    def backward(self, dL_dphiN, want_da=False):
        """Gradients of the last forward_ckpt: (dL/dphi0, dL/dD (numpy), dL/ds (numpy), dL/da or None)."""
        g = dL_dphiN.to(self.device, torch.float32).contiguous()
        dphi0 = torch.empty(self.shape, device=self.device, dtype=torch.float32)
        dD = np.zeros(self.dim * self.dim)
        ds = np.zeros(15)
        da = torch.empty((self.dim,) + self.shape, device=self.device, dtype=torch.float32) if want_da else None
        self._ck(self.L.lbm_cde_backward(self.h, g.data_ptr(), dphi0.data_ptr(), dD.ctypes.data_as(N._DP),
                                         ds.ctypes.data_as(N._DP), da.data_ptr() if da is not None else None),
                 "lbm_cde_backward")
        return dphi0, dD.reshape(self.dim, self.dim), ds, da

    def set_profiling(self, on=True):
        """Per-phase device timing of later backward() sweeps (backward_phases())."""
        self._ck(self.L.lbm_cde_set_profiling(self.h, 1 if on else 0), "lbm_cde_set_profiling")

    def backward_phases(self):
        """(recompute ms, reverse steps ms, whole sweep ms) of the last profiled backward()."""
        v = np.zeros(3)
        self._ck(self.L.lbm_cde_backward_phases(self.h, v.ctypes.data_as(N._DP)), "lbm_cde_backward_phases")
        return {"recompute_ms": float(v[0]), "reverse_steps_ms": float(v[1]), "sweep_ms": float(v[2])}

    def run_host(self, phi0: np.ndarray, nsteps: int, out: np.ndarray | None = None):
        phi0 = np.ascontiguousarray(phi0, dtype=np.float32)
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        self._ck(self.L.lbm_cde_run_host(self.h, phi0.ctypes.data, int(nsteps), out.ctypes.data),
                 "lbm_cde_run_host")
        return out
