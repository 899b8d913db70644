"""GB300 (sm_103a) modified-MRT lattice Boltzmann solver for the
convection-diffusion equation (Huang & Wu, arXiv:1404.2363).

The compute path is liblbm_cde.so (hand-written CUDA behind the C ABI of
include/lbm_cde.h); ``_native`` is its ctypes binding and ``Solver`` a
torch-facing convenience wrapper. ``workloads`` builds the seeded synthetic
inputs.
"""
from . import _native  # noqa: F401

__all__ = ["Solver", "lib"]


def lib():
    return _native.lib()


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver

        return Solver
    raise AttributeError(name)
