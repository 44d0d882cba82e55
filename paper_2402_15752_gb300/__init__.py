"""GB300-native phase-field lattice Boltzmann with interfacial mass/heat transfer.

The solver is the C-ABI library liblbm (include/lbm.h, CUDA for sm_103a);
``Simulation`` is its Python binding and ``Batch`` groups simulations for the
batched runner.  ``workloads`` generates the seeded
synthetic inputs.  Importing the package does not load the library; the first
``Simulation`` does, and raises if it has not been built.
"""
from .batch import Batch  # noqa: F401
from .lbm import (FIELDS, LBMError, Simulation, load_library, make_params,  # noqa: F401
                  workspace_bytes)
