"""FP64 CPU oracle for the modified-MRT lattice Boltzmann model (arXiv:1404.2363).

TEST INFRASTRUCTURE. Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package. The GPU library never imports it and shares no code with it.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, optional OpenMP over
cells); this module loads it with ctypes, drives the time loop, and holds the
closed forms the paper states:

* the D <-> A relation of Eq. 36 (D2Q9) and Eq. A.6 (D3Q15),
* the Gaussian-hill solution of Eq. 40-41,
* the error norms of Eq. 43 and Eq. 45,
* the Taylor-Aris estimator of Eq. 46-49.

Parity status per function is listed in ``PINS`` below; every function is
pinned by a test under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

MRT_A, MRT_B1, MRT_B2, MRT_B3 = 0, 1, 2, 3
PERIODIC, NOFLUX_NODE, BOUNCEBACK, DIRICHLET = 0, 1, 2, 3

PINS = {
    "tables (e, M, M^-1, S)": "tests/test_oracle_tables.py",
    "collision": "tests/test_oracle_collision.py",
    "step / streaming / walls": "tests/test_oracle_step.py",
    "Gaussian hill (Eq. 41, Tables 1-2)": "tests/test_oracle_gaussian.py",
    "Taylor-Aris (Eq. 46-49, Tables 3-5)": "tests/test_oracle_taylor_aris.py",
    "adjoint": "tests/test_oracle_adjoint.py",
    "D3Q15": "tests/test_oracle_d3q15.py",
}


def build(force: bool = False) -> str:
    """Compiles lbm_oracle.c into liblbm_oracle.so (gcc, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int32),
        ("model", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("bc_lo", ctypes.c_int32),
        ("bc_hi", ctypes.c_int32),
        ("phi_w_lo", ctypes.c_double),
        ("phi_w_hi", ctypes.c_double),
        ("alpha1", ctypes.c_double),
        ("alpha2", ctypes.c_double),
        ("s", ctypes.c_double * 15),
        ("A", ctypes.c_double * 9),
        ("nthreads", ctypes.c_int32),
        ("bcx_lo", ctypes.c_int32),
        ("bcx_hi", ctypes.c_int32),
        ("bcz_lo", ctypes.c_int32),
        ("bcz_hi", ctypes.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        _lib.orc_lattice_tables.argtypes = [pp, ctypes.POINTER(ctypes.c_int), dp, dp, dp]
        _lib.orc_meq.argtypes = [pp, ctypes.c_double, dp, dp]
        _lib.orc_collide_node.argtypes = [pp, dp, dp, dp]
        _lib.orc_init_eq.argtypes = [pp, dp, dp, dp]
        _lib.orc_phi.argtypes = [pp, dp, dp]
        _lib.orc_step.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_run.argtypes = [pp, dp, dp, ctypes.c_int64]
        _lib.orc_adjoint_step.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        _lib.orc_feq_jacobian.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_channel_moments.argtypes = [pp, dp, dp, dp, ctypes.c_int64, dp]
        _lib.orc_max_threads.restype = ctypes.c_int
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------

def diffusion_factor(q: int, alpha1: float, alpha2: float, model: int = MRT_A) -> float:
    """The scalar k in D = k dt (I - A/2) A^-1: Eq. 36 for D2Q9, Eq. A.6 for D3Q15.
    The unmodified D2Q9 models MRT-B1/B2/B3 (Sec. 3.1, after Eq. 39) all give
    k = 1/3, whatever constants their equilibria carry."""
    if q == 9 and model != MRT_A:
        return 1.0 / 3.0
    if q == 9:
        return 2.0 / 3.0 + alpha1 / 8.0 + alpha2 / 12.0
    return 2.0 / 3.0 + 55.0 / 54.0 * alpha1 + alpha2 / 216.0


def A_from_D(D, q: int = 9, alpha1: float = -8.0, alpha2: float = 8.0):
    """Inverts D = k (I - A/2) A^-1 (dt = 1): A^-1 = D/k + I/2, A = (A^-1)^-1."""
    D = np.asarray(D, dtype=np.float64)
    k = diffusion_factor(q, alpha1, alpha2)
    if k <= 0:
        raise ValueError("equilibrium parameters give a non-positive diffusion factor")
    dim = D.shape[0]
    return np.linalg.inv(D / k + 0.5 * np.eye(dim))


def D_from_A(A, q: int = 9, alpha1: float = -8.0, alpha2: float = 8.0):
    """Eq. 36 / A.6 with dt = 1."""
    A = np.asarray(A, dtype=np.float64)
    k = diffusion_factor(q, alpha1, alpha2)
    dim = A.shape[0]
    return k * (np.eye(dim) - A / 2.0) @ np.linalg.inv(A)


@dataclass
class Params:
    """One oracle run. ``s`` holds the diagonal rates s_0..s_{q-1}; the entries of
    the flux rows are unused (they come from ``A``). ``tie`` applies the choice of
    Sec. 3.1 / 3.2: s_4 = s_xx, s_6 = s_yy (and s_8 = s_zz in 3D)."""

    q: int = 9
    model: int = MRT_A
    nx: int = 16
    ny: int = 16
    nz: int = 1
    bc_lo: int = PERIODIC
    bc_hi: int = PERIODIC
    phi_w_lo: float = 0.0
    phi_w_hi: float = 0.0
    alpha1: float = -8.0
    alpha2: float = 8.0
    A: np.ndarray = field(default_factory=lambda: np.eye(2))
    s: np.ndarray | None = None
    tie: bool = True
    nthreads: int = 0
    bcx_lo: int = PERIODIC      # x faces: PERIODIC, NOFLUX_NODE or BOUNCEBACK
    bcx_hi: int = PERIODIC
    bcz_lo: int = PERIODIC      # z faces (D3Q15)
    bcz_hi: int = PERIODIC

    @property
    def dim(self) -> int:
        return 2 if self.q == 9 else 3

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def rates(self) -> np.ndarray:
        if self.s is not None:
            s = np.array(self.s, dtype=np.float64).copy()
        elif self.q == 9:
            # Sec. 3.1 (convergence study): s0 = 1, s1 = s2 = 1.1, s7 = s8 = 1.2
            s = np.array([1.0, 1.1, 1.1, 0.0, 1.0, 0.0, 1.0, 1.2, 1.2])
        else:
            s = np.array([1.0, 1.1, 1.1, 0, 1.0, 0, 1.0, 0, 1.0] + [1.2] * 6)
        A = np.asarray(self.A, dtype=np.float64)
        if self.tie:
            s[4] = A[0, 0]
            s[6] = A[1, 1]
            if self.q == 15:
                s[8] = A[2, 2]
        return s

    def c(self) -> _Params:
        p = _Params()
        p.q, p.model = self.q, self.model
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.bc_lo, p.bc_hi = self.bc_lo, self.bc_hi
        p.phi_w_lo, p.phi_w_hi = self.phi_w_lo, self.phi_w_hi
        p.alpha1, p.alpha2 = self.alpha1, self.alpha2
        s = self.rates()
        for k in range(15):
            p.s[k] = float(s[k]) if k < len(s) else 0.0
        A = np.asarray(self.A, dtype=np.float64).reshape(-1)
        for k in range(9):
            p.A[k] = float(A[k]) if k < len(A) else 0.0
        p.nthreads = self.nthreads
        p.bcx_lo, p.bcx_hi = self.bcx_lo, self.bcx_hi
        p.bcz_lo, p.bcz_hi = self.bcz_lo, self.bcz_hi
        return p


def default_params_3d(**kw) -> Params:
    """D3Q15 defaults: alpha1 = -6/5, alpha2 = 192 (the paper leaves them open;
    these make the A.6 factor 1/3 and cancel the q-flux contribution)."""
    kw.setdefault("q", 15)
    kw.setdefault("alpha1", -6.0 / 5.0)
    kw.setdefault("alpha2", 192.0)
    kw.setdefault("A", np.eye(3))
    return Params(**kw)


# ---------------------------------------------------------------------------
# Wrappers
# ---------------------------------------------------------------------------

def tables(p: Params):
    q = p.q
    e = np.zeros(q * 3, dtype=np.int32)
    M = np.zeros(q * q)
    Mi = np.zeros(q * q)
    S = np.zeros(q * q)
    c = p.c()
    _check(lib().orc_lattice_tables(ctypes.byref(c), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    _dp(M), _dp(Mi), _dp(S)), "tables")
    return e.reshape(q, 3), M.reshape(q, q), Mi.reshape(q, q), S.reshape(q, q)


def meq(p: Params, phi: float, u) -> np.ndarray:
    out = np.zeros(p.q)
    uu = np.zeros(3)
    uu[: len(u)] = u
    c = p.c()
    _check(lib().orc_meq(ctypes.byref(c), float(phi), _dp(uu), _dp(out)), "meq")
    return out


def collide_node(p: Params, f, u) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(p.q)
    uu = np.zeros(3)
    uu[: len(u)] = u
    c = p.c()
    _check(lib().orc_collide_node(ctypes.byref(c), _dp(f), _dp(uu), _dp(out)), "collide")
    return out


def _u_arr(p: Params, u):
    if u is None:
        return None
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(p.dim, p.ncell))
    return u


def init_eq(p: Params, phi, u=None) -> np.ndarray:
    """f(0) = f^eq(phi_0, u(0)) = M^-1 m^eq (the initialisation reading)."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
    f = np.zeros(p.q * p.ncell)
    ua = _u_arr(p, u)
    c = p.c()
    _check(lib().orc_init_eq(ctypes.byref(c), _dp(phi), _dp(ua), _dp(f)), "init_eq")
    return f


def phi_of(p: Params, f) -> np.ndarray:
    out = np.zeros(p.ncell)
    c = p.c()
    _check(lib().orc_phi(ctypes.byref(c), _dp(f), _dp(out)), "phi")
    return out


def step(p: Params, f, u=None, scratch=None) -> np.ndarray:
    ua = _u_arr(p, u)
    post = scratch if scratch is not None else np.empty_like(f)
    out = np.empty_like(f)
    c = p.c()
    _check(lib().orc_step(ctypes.byref(c), _dp(f), _dp(ua), _dp(post), _dp(out)), "step")
    return out


def run(p: Params, phi0, nsteps: int, u=None, u_of_t=None, return_f: bool = False):
    """Initialises at equilibrium and runs ``nsteps`` steps. ``u_of_t(t)`` (if
    given) returns the velocity used by the collision at time t, t = 0 .. n-1,
    and the initial state uses u_of_t(0)."""
    if u_of_t is None:
        f = init_eq(p, phi0, u)
        if nsteps > 0:
            c = p.c()
            _check(lib().orc_run(ctypes.byref(c), _dp(f), _dp(_u_arr(p, u)), int(nsteps)), "run")
    else:
        f = init_eq(p, phi0, u_of_t(0))
        post = np.empty_like(f)
        for t in range(nsteps):
            f = step(p, f, u_of_t(t), post)
    phi = phi_of(p, f)
    return (phi, f) if return_f else phi


def adjoint_step(p: Params, lam_next, f_pre, u=None, want_dS=False, want_du=False):
    ua = _u_arr(p, u)
    lam = np.empty_like(lam_next)
    dS = np.zeros(p.q * p.q) if want_dS else None
    du = np.zeros(p.dim * p.ncell) if want_du else None
    c = p.c()
    _check(lib().orc_adjoint_step(ctypes.byref(c), _dp(lam_next), _dp(f_pre), _dp(ua), _dp(lam),
                                  _dp(dS), _dp(du)), "adjoint_step")
    return lam, (dS.reshape(p.q, p.q) if dS is not None else None), du


def feq_jacobian(p: Params, phi, u=None):
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
    dphi = np.zeros(p.q * p.ncell)
    du = np.zeros(p.dim * p.q * p.ncell)
    c = p.c()
    _check(lib().orc_feq_jacobian(ctypes.byref(c), _dp(phi), _dp(_u_arr(p, u)), _dp(dphi), _dp(du)),
           "feq_jacobian")
    return dphi, du


def channel_moments(p: Params, ux_row, F0, wy, nsteps: int) -> np.ndarray:
    ux_row = np.ascontiguousarray(ux_row, dtype=np.float64)
    F0 = np.ascontiguousarray(F0, dtype=np.float64).reshape(-1)
    wy = np.ascontiguousarray(wy, dtype=np.float64)
    out = np.zeros((nsteps + 1) * 3)
    c = p.c()
    _check(lib().orc_channel_moments(ctypes.byref(c), _dp(ux_row), _dp(F0), _dp(wy), int(nsteps),
                                     _dp(out)), "channel_moments")
    return out.reshape(nsteps + 1, 3)


# ---------------------------------------------------------------------------
# Adjoint driver (reverse sweep with every forward state kept; small cases)
# ---------------------------------------------------------------------------

def s_gradients(p: Params, dS: np.ndarray) -> dict:
    """Chain rule from dL/dS (per entry) to the named relaxation parameters.
    D2Q9 MRT-A (Eq. 31): S33 = sxx, S34 = (sxx/2 - 1) s4, S35 = sxy, S36 = sxy/2 s6,
    S53 = syx, S54 = syx/2 s4, S55 = syy, S56 = (syy/2 - 1) s6, S44 = s4, S66 = s6."""
    assert p.q == 9
    A = np.asarray(p.A, dtype=np.float64)
    s = p.rates()
    s4, s6 = s[4], s[6]
    g = {}
    mod = p.model == MRT_A
    g["sxx"] = dS[3, 3] + (0.5 * s4 * dS[3, 4] if mod else 0.0)
    g["sxy"] = dS[3, 5] + (0.5 * s6 * dS[3, 6] if mod else 0.0)
    g["syx"] = dS[5, 3] + (0.5 * s4 * dS[5, 4] if mod else 0.0)
    g["syy"] = dS[5, 5] + (0.5 * s6 * dS[5, 6] if mod else 0.0)
    g["s4"] = dS[4, 4] + ((A[0, 0] / 2 - 1) * dS[3, 4] + A[1, 0] / 2 * dS[5, 4] if mod else 0.0)
    g["s6"] = dS[6, 6] + (A[0, 1] / 2 * dS[3, 6] + (A[1, 1] / 2 - 1) * dS[5, 6] if mod else 0.0)
    return g


def grad_D_from_s(p: Params, gs: dict) -> np.ndarray:
    """dL/dD for the parametrisation A = (D/k + I/2)^-1 with s4 = sxx, s6 = syy
    (tie) and S symmetric in the off-diagonal block (sxy = syx = A01)."""
    A = np.asarray(p.A, dtype=np.float64)
    k = diffusion_factor(p.q, p.alpha1, p.alpha2, p.model)
    GA = np.array([[gs["sxx"] + (gs["s4"] if p.tie else 0.0), gs["sxy"]],
                   [gs["syx"], gs["syy"] + (gs["s6"] if p.tie else 0.0)]])
    # dA = -A (dD / k) A  =>  dL/dD = -(1/k) A^T GA A^T
    return -(A.T @ GA @ A.T) / k


# ---------------------------------------------------------------------------
# Closed forms of the paper
# ---------------------------------------------------------------------------

def gaussian_hill(X, Y, t, D, u, sigma0, phi0_total, images: int = 1, L=None):
    """Eq. 41: phi = phi0 / (2 pi sqrt(det sigma_t)) exp(-1/2 sigma_t^-1 : (x - u t)(x - u t)),
    sigma_t = sigma0^2 I + 2 t D. With ``L`` (box lengths) the periodic images
    within +-``images`` boxes are summed."""
    D = np.asarray(D, dtype=np.float64)
    st = sigma0 ** 2 * np.eye(2) + 2.0 * t * D
    si = np.linalg.inv(st)
    pref = phi0_total / (2.0 * math.pi * math.sqrt(np.linalg.det(st)))
    out = np.zeros_like(X, dtype=np.float64)
    shifts = range(-images, images + 1) if L is not None else [0]
    for a in shifts:
        for b in shifts:
            dx = X - u[0] * t - (a * L[0] if L is not None else 0.0)
            dy = Y - u[1] * t - (b * L[1] if L is not None else 0.0)
            qf = si[0, 0] * dx * dx + 2 * si[0, 1] * dx * dy + si[1, 1] * dy * dy
            out += pref * np.exp(-0.5 * qf)
    return out


def er2(num, ana):
    """Eq. 43 (average error)."""
    return float(np.sqrt(np.mean((num - ana) ** 2)))


def er_inf(num, ana):
    """Eq. 43 (maximum error)."""
    return float(np.max(np.abs(num - ana)))


def er_rel(num, ana):
    """Eq. 45 (relative error)."""
    return float(np.sqrt(np.sum((num - ana) ** 2)) / np.sqrt(np.sum(ana ** 2)))


def taylor_aris_analytic(alpha: float, Pe: float) -> float:
    """alpha_L = alpha (1 + Pe^2 / 210) (Sec. 3.2)."""
    return alpha * (1.0 + Pe * Pe / 210.0)


def variance_from_moments(mom):
    """Eq. 47 from the running sums (sum phi, sum x phi, sum x^2 phi)."""
    m0, m1, m2 = mom[..., 0], mom[..., 1], mom[..., 2]
    return m2 / m0 - (m1 / m0) ** 2


def alpha_series(mom):
    """Discrete Eq. 46: alpha_n = (sigma^2_{n+1} - sigma^2_n) / 2."""
    s2 = variance_from_moments(mom)
    return 0.5 * np.diff(s2)


def converged_alpha(alpha_n, window: int = 100, tol: float = 1e-6):
    """Eq. 49 (with |.|): first n with |a_{n+window} - a_n| / a_n <= tol."""
    a = np.asarray(alpha_n)
    for n in range(len(a) - window):
        if abs(a[n + window] - a[n]) / a[n] <= tol:
            return n, float(a[n])
    return None, float(a[-1])


def adjoint_gradients(p: Params, phi0, nsteps: int, dL_dphiN, u=None, u_of_t=None):
    """Reverse sweep of ``run`` keeping every forward state (small grids only).
    The velocity is ``u`` (constant in time) or ``u_of_t(t)``. Returns
    (dL/dphi0 [ncell], dL/dD [dim x dim, entries treated independently],
     dL/du [nsteps][dim x ncell] per collision time t (t = 0 includes the
     dependence of the initial equilibrium on u(0)), dL/dS [q x q]). With a
     Dirichlet wall dL/du is not formed (None): the fill's weights depend on u."""
    uf = (lambda t: _u_arr(p, u)) if u_of_t is None else (lambda t: _u_arr(p, u_of_t(t)))
    states = [init_eq(p, phi0, uf(0))]
    post = np.empty_like(states[0])
    for t in range(nsteps):
        states.append(step(p, states[-1], uf(t), post))
    lam = np.tile(np.asarray(dL_dphiN, dtype=np.float64).reshape(-1), p.q)
    dS = np.zeros((p.q, p.q))
    du = np.zeros((max(nsteps, 1), p.dim * p.ncell))
    want_du = DIRICHLET not in (p.bc_lo, p.bc_hi)
    for n in range(nsteps - 1, -1, -1):
        lam, dSn, dun = adjoint_step(p, lam, states[n], uf(n), want_dS=True, want_du=want_du)
        dS += dSn
        if want_du:
            du[n] += dun
    dphi, dfdu = feq_jacobian(p, phi0, uf(0))
    lam2 = lam.reshape(p.q, p.ncell)
    g_phi0 = (lam2 * dphi.reshape(p.q, p.ncell)).sum(axis=0)
    du[0] += (dfdu.reshape(p.dim, p.q, p.ncell) * lam2[None]).sum(axis=1).reshape(-1)
    gD = grad_D_from_s(p, s_gradients(p, dS)) if p.q == 9 else None
    if not want_du:
        return g_phi0, gD, None, dS
    if u_of_t is None:
        return g_phi0, gD, du.sum(axis=0).reshape(p.dim, p.ncell), dS
    return g_phi0, gD, du.reshape(-1, p.dim, p.ncell), dS
