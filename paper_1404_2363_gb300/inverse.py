"""Inverse problem through the hand-written adjoint: recover the diffusion
tensor D and the low Fourier modes of the initial field phi0 of Eq. 1 from
noisy snapshots phi(x, t_k) of a D2Q9 MRT-A run.

Parametrisation (the unknowns the optimiser sees):
  D    = L L^T with L = [[exp t0, 0], [t1, exp t2]]   (every trial point SPD)
  phi0 = base + Re IFFT2(C)  (orthonormal transform; C is zero outside the
         modes x modes block of wave numbers kx, ky in [-modes/2, modes/2))
The misfit L = sum_k sum_x (phi(x, t_k; D, phi0) - obs_k(x))^2 is minimised
with torch L-BFGS; each evaluation runs one lbm_cde_forward_ckpt (sqrt(N)
checkpoints) and one lbm_cde_backward per segment through ``autograd.lbm_run``.
The Fourier maps are plain torch operations on the parameters, outside the
solver's hot path.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .autograd import lbm_run


def mode_index(n: int, modes: int, device=None):
    """Flat indices (ky mod n) * n + (kx mod n) of the modes x modes block."""
    h = modes // 2
    k = torch.arange(-h, h, device=device) % n
    return (k[:, None] * n + k[None, :]).reshape(-1)


def field_from_modes(C: torch.Tensor, n: int, idx: torch.Tensor) -> torch.Tensor:
    """Re IFFT2 (orthonormal) of the block coefficients C = (2, modes, modes)
    (real and imaginary parts) placed at idx in an n x n spectrum."""
    spec = torch.zeros(n * n, dtype=torch.complex128, device=C.device)
    spec = spec.index_put((idx,), torch.complex(C[0].reshape(-1), C[1].reshape(-1)))
    return torch.fft.ifft2(spec.reshape(n, n), norm="ortho").real


def modes_from_field(f: torch.Tensor, modes: int) -> torch.Tensor:
    """Block coefficients whose field_from_modes reproduces the projection of f
    onto the block's real modes (the Hermitian-symmetric part of its spectrum)."""
    n = f.shape[-1]
    idx = mode_index(n, modes, f.device)
    spec = torch.fft.fft2(f.to(torch.float64), norm="ortho").reshape(-1)
    c = spec[idx]
    return torch.stack([c.real, c.imag]).reshape(2, modes, modes)


def project(f: torch.Tensor, modes: int) -> torch.Tensor:
    """Projection of a real field onto the real span of the block's modes."""
    n = f.shape[-1]
    idx = mode_index(n, modes, f.device)
    spec = torch.fft.fft2(f.to(torch.float64), norm="ortho").reshape(-1)
    keep = torch.zeros(n * n, dtype=torch.bool, device=f.device)
    keep[idx] = True
    # the conjugate partners -k of the block carry the same real modes
    ky, kx = idx // n, idx % n
    keep[((-ky) % n) * n + (-kx) % n] = True
    return torch.fft.ifft2(torch.where(keep, spec, torch.zeros_like(spec)).reshape(n, n), norm="ortho").real


def D_of(theta: torch.Tensor) -> torch.Tensor:
    l00, l10, l11 = torch.exp(theta[0]), theta[1], torch.exp(theta[2])
    return torch.stack([torch.stack([l00 * l00, l00 * l10]),
                        torch.stack([l00 * l10, l10 * l10 + l11 * l11])])


def theta_of(D) -> torch.Tensor:
    Lc = np.linalg.cholesky(np.asarray(D, dtype=np.float64))
    return torch.tensor([math.log(Lc[0, 0]), Lc[1, 0], math.log(Lc[1, 1])], dtype=torch.float64)


def recover(solvers, observations, a: torch.Tensor, modes: int = 64, D0=None, base: float = 1.0,
            sched=None, fit_D: bool = True, fit_phi0: bool = True, D_fixed=None, phi0_fixed=None,
            max_iter: int = 200, every: int = 0, history: int = 50):
    """Minimises the snapshot misfit sum_k sum_x (phi(x, t_k) - obs_k(x))^2 over
    (D, phi0 modes), starting from D0 (default 0.03 I) and phi0 = base.

    observations: list of (t_k, obs_k) with increasing t_k (steps) and obs_k an
    (n, n) tensor. solvers: one paper_1404_2363_gb300.Solver (FP32 storage, the
    grid of obs) per observation; segment k runs from t_{k-1} to t_k on
    solvers[k] (each keeps the checkpoints of its own segment for the reverse
    sweep). fit_D / fit_phi0 = False hold D at D_fixed or phi0 at phi0_fixed.
    Returns a dict with the estimates, the final misfit and the evaluation count.

    One final snapshot alone does not determine D and phi0 together: a smaller
    D with a correspondingly smoother phi0 (each mode scaled by the decay the
    missing diffusion would have caused) gives nearly the same phi(t_N) (exactly
    so for a constant velocity, where advection and diffusion commute), so the
    misfit reaches the noise level along that whole family. A second snapshot
    (or a known phi0 or D) removes the freedom."""
    obs0 = observations[0][1]
    n = obs0.shape[-1]
    dev = obs0.device
    idx = mode_index(n, modes, dev)
    theta0 = theta_of(np.eye(2) * 0.03 if D0 is None else D0).to(dev)
    # the optimiser moves psi = (theta - theta0) * w: w is the square root of the
    # Gauss-Newton curvature of the misfit along each theta entry (relative to the
    # mode coefficients, whose curvature is about 1 per snapshot), so that one
    # L-BFGS history serves both kinds of unknowns
    w = torch.ones(3, dtype=torch.float64, device=dev)
    psi = torch.zeros(3, dtype=torch.float64, device=dev, requires_grad=fit_D)
    C = torch.zeros((2, modes, modes), dtype=torch.float64, device=dev, requires_grad=fit_phi0)
    evals = [0]
    Dfix = None if D_fixed is None else torch.as_tensor(np.asarray(D_fixed), dtype=torch.float64, device=dev)
    lo = torch.tensor([0.5 * math.log(1e-5), -1.0, 0.5 * math.log(1e-5)], dtype=torch.float64, device=dev)
    hi = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64, device=dev)

    def theta():
        # kept in a box (D entries between 1e-5 and 1) so that no trial point of
        # a line search gives a non-finite or unstable D
        return torch.minimum(torch.maximum(theta0 + psi / w, lo), hi)

    def model(th=None):
        phi = (base + field_from_modes(C, n, idx)).to(torch.float32) if fit_phi0 else phi0_fixed.to(torch.float32)
        D = D_of(theta() if th is None else th) if fit_D else Dfix
        out, t_prev = [], 0
        for s, (t, _) in zip(solvers, observations):
            sk = None if sched is None else torch.roll(sched, -t_prev, dims=0)
            phi = lbm_run(phi, D, a, solver=s, nsteps=t - t_prev, sched=sk, every=every)
            out.append(phi)
            t_prev = t
        return out

    def misfit():
        return sum(((p.to(torch.float64) - o.to(torch.float64)) ** 2).sum()
                   for p, (_, o) in zip(model(), observations))

    def run(params, iters):
        opt = torch.optim.LBFGS(params, lr=1.0, max_iter=iters, history_size=history,
                                tolerance_grad=1e-12, tolerance_change=1e-14, line_search_fn="strong_wolfe")

        def closure():
            opt.zero_grad()
            loss = misfit()
            loss.backward()
            evals[0] += 1
            return loss

        opt.step(closure)

    def rescale():
        # forward differences of the model along each theta entry
        with torch.no_grad():
            th = theta()
            ref = [p.to(torch.float64) for p in model(th)]
            for i in range(3):
                h = 1e-2
                tp = th.clone()
                tp[i] += h
                j2 = sum(float((((q.to(torch.float64) - r) / h) ** 2).sum()) for q, r in zip(model(tp), ref))
                wi = math.sqrt(max(j2 / len(observations), 1.0))
                psi[i] = (th[i] - theta0[i]) * wi
                w[i] = wi

    if fit_D and fit_phi0:
        run([C], max_iter // 4)          # modes first: at phi0 = base, phi(t) does not depend on D
        for _ in range(2):
            rescale()
            run([psi, C], max_iter // 2)
    elif fit_D:
        rescale()
        run([psi], max_iter)
    else:
        run([C], max_iter)
    with torch.no_grad():
        phi0 = base + field_from_modes(C, n, idx) if fit_phi0 else phi0_fixed.to(torch.float64)
        loss = float(misfit().item())
    D = D_of(theta()).detach().cpu().numpy() if fit_D else np.asarray(D_fixed, dtype=np.float64)
    return {"D": D, "phi0": phi0, "C": C.detach(), "loss": loss, "evaluations": evals[0]}
