"""GB300 (sm_103a) relativistic lattice Boltzmann step for finite-mass
particles (Gabbana, Mendoza, Succi & Tripiccione, arXiv:1703.04605).

The method runs in librlbm.so (C ABI, include/rlbm.h): hand-written CUDA
kernels for the fused pull-stream / moments / Landau frame / EOS /
equilibrium / Anderson-Witting collision step.  This package only marshals
arguments; it has no host implementation of the step."""
from . import _abi
from ._abi import RLBMError, load, quadrature_weights, quadrature_window, bessel_ratio
from .lattice import (Lattice, Lattice3D, batch_engine, batch_step, batch_tuning, set_batch_options, use_cuda_malloc,
                      use_torch_allocator)

__all__ = ["Lattice", "Lattice3D", "batch_step", "batch_tuning", "batch_engine", "set_batch_options",
           "use_torch_allocator", "use_cuda_malloc", "RLBMError", "load", "quadrature_weights", "quadrature_window",
           "bessel_ratio"]
