"""Plain, slow FP64 CPU oracle of the moment-represented lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check in __graft_entry__ and the CPU
baseline legs of bench.py may import this package. The library (paper_2609_09160_gb300) never
imports it and shares no code with it; the two meet only through the seeded input generators
of the `synth` package, which hold none of the method's arithmetic.

Modules
  lattice      D3Q19 / D3Q27 velocity sets, the second-order Hermite basis (textbook values) and
               the complete D3Q27 Hermite basis of D3Q27h
  lbm          population-form step: Hermite projection, Eq. (corr), regularized collision with
               Guo forcing, Eq. (pullLB), pull streaming with halfway bounce-back
  moment_form  literal site-by-site transcription of Eq. (pullLLB) + Eq. (corr), tiny lattices
  phase        conservative Allen-Cahn FTCS, chemical potential, capillary force, two-component run
  adjoint      gradients of one step and of a rollout loss (autograd of lbm)
  diagnostics  FP64 reductions and the closed forms the tests compare against

Parity status: every function is pinned by tests/test_oracle_*.py against closed forms,
invariants, textbook identities, brute force or finite differences; none is "parity unpinned".
"""
from . import adjoint, diagnostics, lattice, lbm, moment_form, phase  # noqa: F401
from .lattice import CS2, D3Q19, D3Q27, D3Q27H  # noqa: F401
