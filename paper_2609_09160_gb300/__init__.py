"""GB300-native moment-represented lattice Boltzmann step (arXiv 2609.09160, Sec. 2).

liblbf.so (CUDA, sm_103a) holds every step of the method; this package is its Python binding:
`_lbf` mirrors the C ABI of include/lbf.h function by function, `Solver` owns a context and its
torch-allocated workspace, and `Rollout` is the autograd Function built on the adjoint kernel.
The library must be built (`python -m paper_2609_09160_gb300.build`); nothing falls back to
the CPU.
"""
from . import _lbf  # noqa: F401
from ._lbf import LBFError, load_library  # noqa: F401
from .rollout import Rollout, rollout  # noqa: F401
from .solver import Solver  # noqa: F401
