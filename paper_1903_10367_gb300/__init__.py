"""GB300-native adAFAC: additively damped asynchronous fast adaptive composite
multigrid (Murray & Weinzierl, arXiv:1903.10367) as hand-written sm_103a CUDA
kernels behind a C ABI (include/adafac.h).

``paper_1903_10367_gb300.adafac`` is the thin Python binding; importing this
package does not load or build the library (``adafac.load()`` does, and fails
loudly when it cannot).
"""
from .adafac import (AdafacError, Options, Solver, Tree, default_options, load,  # noqa: F401
                     workspace_size)
