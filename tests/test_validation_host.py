"""Host-side pins of the validation helpers (no GPU): the device closed form of
Eq. 41 and t_m against the oracle's independent versions, and the Eq. 44
matrices against the Table 1 full-anisotropic case."""
import math

import numpy as np
import torch
from scipy.optimize import brentq

from paper_1404_2363_gb300 import validation as V


def test_t_m_closed_root_matches_bracketing():
    for D in (V.lattice_D(V.EQ42["iso"]), V.lattice_D(V.EQ42["full"]), V.eq44_D("diag", 1.3)):
        want = brentq(lambda t: np.linalg.det(12.8 ** 2 * np.eye(2) + 2 * t * D) - 4 * 12.8 ** 4, 1e-6, 1e7)
        assert abs(V.t_m(D, 12.8) - want) < 1e-9 * want
    # isotropic: (sigma0^2 + 2 t D)^2 = 4 sigma0^4  =>  t = sigma0^2 / (2 D)
    assert abs(V.t_m(0.0512 * np.eye(2), 12.8) - 1600.0) < 1e-9


def test_eq44_full_tau_reproduces_table1_full_matrix():
    """Eq. 44's full matrix at tau = 0.5768 is Eq. 42's full D on dx = 1/256."""
    assert np.allclose(V.eq44_D("full", 0.5768), V.lattice_D(V.EQ42["full"]), atol=1e-12)
    assert np.allclose(V.eq44_D("iso", 0.6536), V.lattice_D(V.EQ42["iso"]), atol=1e-12)


def test_exact_matches_oracle_closed_form(O):
    for u in ((0.0, 0.0), (0.05, 0.05)):
        h = V.Hill(N=96, D=np.array([[0.03, 0.01], [0.01, 0.05]]), u=u, sigma0=5.0, steps=700)
        got = h.exact("cpu").numpy()
        j = np.arange(96) - 48
        X, Y = np.meshgrid(j.astype(float), j.astype(float), indexing="xy")
        want = O.gaussian_hill(X, Y, 700, h.D, u, 5.0, 2 * math.pi * 25.0, images=1, L=[96, 96])
        assert np.abs(got - want).max() < 1e-14


def test_errors_definitions(O):
    g = torch.Generator().manual_seed(3)
    a = torch.rand(17, 19, generator=g, dtype=torch.float64)
    b = a + 1e-3 * torch.randn(17, 19, generator=g, dtype=torch.float64)
    e = V.errors(b.float(), a)
    bn, an = b.float().double().numpy(), a.numpy()
    assert abs(e["er2"] - O.er2(bn, an)) < 1e-15
    assert abs(e["er_inf"] - O.er_inf(bn, an)) < 1e-15
    assert abs(e["er_rel"] - O.er_rel(bn, an)) < 1e-15
