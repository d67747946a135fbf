"""GB300-native (sm_103a) single-relaxation-time D2Q9 lattice Boltzmann method
for wave propagation in isotropic linear elastic solids (arXiv 2009.06404).

The time step runs in the CUDA library built from ``csrc/`` (C ABI declared in
``include/lbm_elastic.h``); ``binding`` wraps it with ctypes and uses PyTorch
only for device memory and streams.  ``workloads`` builds seeded synthetic
inputs.
"""
from .binding import (SYMBOLS, Adjoint, Batch, ElasticLBM, LBMError, NonFiniteError, from_workload,
                      load_library, make_config)

__all__ = ["Adjoint", "Batch", "ElasticLBM", "LBMError", "NonFiniteError", "from_workload",
           "load_library", "make_config", "SYMBOLS"]
