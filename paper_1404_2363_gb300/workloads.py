"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds inputs (initial fields, velocity fields, diffusion
tensors, instance lists). It holds none of the lattice Boltzmann arithmetic,
and both the GPU tests and the oracle tests draw their inputs from it.

Recipes (numpy PCG64, seed = 20140409 + workload number):

1. Anisotropic Gaussian hill (Sec. 3.1 shape): periodic n x n, u = 0,
   D = [[0.02, 0.01], [0.01, 0.04]], phi0 = exp(-|x - x0|^2 / (2 * 10^2)),
   x0 on the central node.
2. Gaussian hill in a space- and time-varying velocity: periodic n x n,
   u(x, t) = U0 (sin(2 pi y / n) cos(w t), sin(2 pi x / n) sin(w t)),
   U0 = 0.05, w = 2 pi / 2000, stored as a static field
   a(x) = U0 (sin(2 pi y / n), sin(2 pi x / n)) times a per-step schedule
   (cos w t, sin w t). D = (tau - 1/2)/3 [[1, 1], [1, 4]] (the full
   anisotropic family of Eq. 44), sigma0 = 0.025 n at the centre.
3. Taylor-Aris channel batch (Sec. 3.2 shape): uneven nx in [2048, 8192]
   (periodic), ny in [32, 128] nodes with walls on the nodes, Pe log-uniform
   in [10, 200], U = 0.1, tau = 2 U W / Pe + 1/2 (W = ny - 1) kept in
   [0.55, 2.5] by rescaling U within [0.02, 0.2] or resampling; Poiseuille
   u_x = 4 U y (W - y) / W^2 per row; pulse phi = 1 on columns with
   x / nx in [0.197, 0.203].
4. D3Q15 Gaussian hill: periodic n^3, D = Q diag(lambda) Q^T with
   lambda ~ U[0.01, 0.05] and Q a seeded rotation, u = curl(psi) with psi a
   random Fourier series of integer wave-vectors |k|_inf <= 4, scaled so
   max |u| = 0.05, sigma0 = 0.025 n at the centre.
5. Inverse problem: periodic n x n, u = curl of a seeded stream function
   with 8 x 8 modes scaled to max |u| = 0.05, D_true = [[0.02, 0.01],
   [0.01, 0.04]], phi0 = 1 + a random real Fourier field of 64 x 64 modes,
   amplitude 0.1, k^-2 decay.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED0 = 20140409


def rng(workload: int, extra: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED0 + workload + 1000 * extra))


# ---------------------------------------------------------------------------
# 1. Gaussian hill, u = 0
# ---------------------------------------------------------------------------

D_ANISO = np.array([[0.02, 0.01], [0.01, 0.04]])


def gaussian_phi0(nx: int, ny: int, sigma: float, x0=None, amp: float = 1.0) -> np.ndarray:
    """phi0[y, x] = amp * exp(-|x - x0|^2 / (2 sigma^2)), float64, shape (ny, nx)."""
    if x0 is None:
        x0 = (nx // 2, ny // 2)
    X, Y = np.meshgrid(np.arange(nx) - x0[0], np.arange(ny) - x0[1], indexing="xy")
    return amp * np.exp(-(X * X + Y * Y) / (2.0 * sigma * sigma))


def gaussian_workload(n: int = 128):
    return {"phi0": gaussian_phi0(n, n, 10.0), "D": D_ANISO.copy(), "u": None}


# ---------------------------------------------------------------------------
# 2. Time-varying vortex velocity
# ---------------------------------------------------------------------------

OMEGA = 2.0 * math.pi / 2000.0
U0 = 0.05


def vortex_field(n: int, U: float = U0) -> np.ndarray:
    """a(x) of shape (2, n, n): a_x = U sin(2 pi y / n), a_y = U sin(2 pi x / n)."""
    j = np.arange(n)
    X, Y = np.meshgrid(j, j, indexing="xy")
    return np.stack([U * np.sin(2 * math.pi * Y / n), U * np.sin(2 * math.pi * X / n)])


def vortex_schedule(nsteps: int, omega: float = OMEGA) -> np.ndarray:
    """(nsteps, 2): multipliers (cos w t, sin w t) for t = 0 .. nsteps-1."""
    t = np.arange(nsteps, dtype=np.float64)
    return np.stack([np.cos(omega * t), np.sin(omega * t)], axis=1)


def D_eq44_full(tau: float) -> np.ndarray:
    """The full anisotropic tensor of Eq. 44 expressed as D: (tau - 1/2)/3 [[1,1],[1,4]]."""
    return (tau - 0.5) / 3.0 * np.array([[1.0, 1.0], [1.0, 4.0]])


def vortex_workload(n: int = 4096, tau: float = 1.0):
    return {
        "phi0": gaussian_phi0(n, n, 0.025 * n),
        "D": D_eq44_full(tau),
        "a": vortex_field(n),
    }


# ---------------------------------------------------------------------------
# 3. Taylor-Aris batch
# ---------------------------------------------------------------------------

@dataclass
class Channel:
    nx: int
    ny: int          # nodes across, walls on nodes 0 and ny-1
    U: float
    tau: float
    Pe: float

    @property
    def W(self) -> int:
        return self.ny - 1

    @property
    def alpha(self) -> float:
        return (self.tau - 0.5) / 3.0

    def ux_row(self) -> np.ndarray:
        y = np.arange(self.ny, dtype=np.float64)
        return 4.0 * self.U * y * (self.W - y) / (self.W * self.W)

    def phi0(self) -> np.ndarray:
        cols = np.arange(self.nx)
        r = cols / self.nx
        pulse = ((r >= 0.197) & (r <= 0.203)).astype(np.float64)
        return np.broadcast_to(pulse, (self.ny, self.nx)).copy()


def taylor_aris_batch(count: int = 64, nx_range=(2048, 8192), ny_range=(32, 128), seed_extra: int = 0):
    g = rng(3, seed_extra)
    out = []
    while len(out) < count:
        nx = int(g.integers(nx_range[0] // 4, nx_range[1] // 4 + 1)) * 4
        ny = int(g.integers(ny_range[0], ny_range[1] + 1))
        Pe = float(math.exp(g.uniform(math.log(10.0), math.log(200.0))))
        W = ny - 1
        U = 0.1
        tau = 2.0 * U * W / Pe + 0.5
        if not (0.55 <= tau <= 2.5):
            U = min(max((np.clip(tau, 0.55, 2.5) - 0.5) * Pe / (2.0 * W), 0.02), 0.2)
            tau = 2.0 * U * W / Pe + 0.5
            if not (0.55 <= tau <= 2.5):
                continue
        out.append(Channel(nx=nx, ny=ny, U=U, tau=tau, Pe=Pe))
    return out


# ---------------------------------------------------------------------------
# 4. D3Q15 Gaussian hill
# ---------------------------------------------------------------------------

def random_rotation(g: np.random.Generator) -> np.ndarray:
    Q, R = np.linalg.qr(g.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def curl_field_3d(n: int, g: np.random.Generator, kmax: int = 4, umax: float = 0.05, shape=None) -> np.ndarray:
    """Divergence-free u = curl(psi), psi a random Fourier vector potential with
    integer wave-vectors |k|_inf <= kmax (per period of each axis); shape
    (3, nz, ny, nx) in [z, y, x] order, nx = ny = nz = n unless shape = (nx, ny, nz)."""
    nx, ny, nz = (n, n, n) if shape is None else shape
    jx, jy, jz = (np.arange(m) * (2.0 * math.pi / m) for m in (nx, ny, nz))
    Z, Y, X = np.meshgrid(jz, jy, jx, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    nmodes = 12
    for _ in range(nmodes):
        k = g.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            continue
        amp = g.standard_normal(3)
        ph = g.uniform(0, 2 * math.pi)
        arg = k[0] * X + k[1] * Y + k[2] * Z + ph
        c = np.cos(arg)
        # curl of amp * sin(arg) = (k x amp) cos(arg)
        # the curl in grid units: d/dx of arg is 2 pi k_x / nx (= k_x 2 pi / n on a cube)
        kg = k.astype(np.float64) * (2.0 * math.pi) / np.array([nx, ny, nz], dtype=np.float64)
        kx = np.cross(kg, amp)
        for a in range(3):
            u[a] += kx[a] * c
    m = np.sqrt((u * u).sum(axis=0)).max()
    return u * (umax / m)


def d3q15_workload(n: int = 384, shape=None):
    """The D3Q15 hill on an n^3 grid, or on nx x ny x nz for shape = (nx, ny, nz)
    (sigma0 = 0.025 of the shortest side)."""
    nx, ny, nz = (n, n, n) if shape is None else shape
    g = rng(4)
    lam = g.uniform(0.01, 0.05, size=3)
    Q = random_rotation(g)
    D = Q @ np.diag(lam) @ Q.T
    u = curl_field_3d(n, g, shape=shape)
    s = 0.025 * min(nx, ny, nz)
    Z, Y, X = np.meshgrid(np.arange(nz) - nz // 2, np.arange(ny) - ny // 2, np.arange(nx) - nx // 2, indexing="ij")
    phi0 = np.exp(-(X * X + Y * Y + Z * Z) / (2 * s * s))
    return {"phi0": phi0, "D": D, "u": u}


# ---------------------------------------------------------------------------
# 5. Inverse problem
# ---------------------------------------------------------------------------

def stream_function_velocity(n: int, g: np.random.Generator, modes: int = 8, umax: float = 0.05):
    """u = (d psi/dy, -d psi/dx) for a random real Fourier psi with modes x modes
    wave-numbers; returns (2, n, n)."""
    j = np.arange(n) * (2.0 * math.pi / n)
    X, Y = np.meshgrid(j, j, indexing="xy")
    ux = np.zeros((n, n))
    uy = np.zeros((n, n))
    for kx in range(-modes // 2, modes // 2 + 1):
        for ky in range(-modes // 2, modes // 2 + 1):
            if kx == 0 and ky == 0:
                continue
            a, b = g.standard_normal(2) / (kx * kx + ky * ky)
            arg = kx * X + ky * Y
            # psi = a cos(arg) + b sin(arg)
            dpsi = -a * np.sin(arg) + b * np.cos(arg)
            ux += ky * dpsi
            uy -= kx * dpsi
    m = np.sqrt(ux * ux + uy * uy).max()
    return np.stack([ux, uy]) * (umax / m)


def fourier_field(n: int, g: np.random.Generator, modes: int = 64, amp: float = 0.1) -> np.ndarray:
    """Real field with (modes x modes) Fourier coefficients ~ N(0,1) k^-2, scaled
    so max |field| = amp; shape (n, n)."""
    c = np.zeros((n, n), dtype=np.complex128)
    h = modes // 2
    for kx in range(-h, h):
        for ky in range(-h, h):
            if kx == 0 and ky == 0:
                continue
            k2 = kx * kx + ky * ky
            c[ky % n, kx % n] = (g.standard_normal() + 1j * g.standard_normal()) / k2
    f = np.fft.ifft2(c).real
    return f * (amp / np.abs(f).max())


def inverse_workload(n: int = 1024, modes: int = 64):
    g = rng(5)
    u = stream_function_velocity(n, g)
    phi0 = 1.0 + fourier_field(n, g, modes=modes)
    return {"phi0": phi0, "D": D_ANISO.copy(), "u": u}


def random_fields(nx: int, ny: int, nz: int = 1, dim: int = 2, seed: int = 0, umax: float = 0.05):
    """Generic random positive phi and bounded u for parity tests (shape-agnostic)."""
    g = rng(0, 17 + seed)
    shape = (nz, ny, nx) if nz > 1 else (ny, nx)
    phi = 0.5 + g.random(shape)
    u = g.uniform(-umax, umax, size=(dim,) + shape)
    return phi, u
