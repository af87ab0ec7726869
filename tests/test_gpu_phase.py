"""GPU parity of the two-component coupling (Allen-Cahn phase field + capillary force, equal
densities) with the FP64 oracle on D3Q19, D3Q27 and D3Q27h, and exact per-component mass
conservation."""
import pytest
import torch

import oracle
import synth
from oracle import phase
from paper_2609_09160_gb300 import Solver

from _helpers import TOL, group_errors, rel_max

pytestmark = pytest.mark.gpu
LAT = {19: oracle.D3Q19, 27: oracle.D3Q27, 127: oracle.D3Q27H}  # 127: D3Q27h
TC = dict(rho_l=1.0, rho_h=1.0, tau_l=1.0, tau_h=0.8, sigma=0.03, width=4.0, diffusivity=0.1)


@pytest.mark.parametrize("lattice", [19, 27, 127])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_two_component_matches_oracle(lattice, storage):
    shape = (14, 17, 35)
    phi0 = synth.droplet(shape, 5.0, 4.0)
    M0 = synth.random_moments(shape, seed=80, p_scale=1e-4, u_scale=1e-3, neq_scale=1e-5)
    s = Solver(shape, lattice=lattice, storage=storage, two_component=TC, force=(1e-6, 0.0, 0.0))
    s.set_moments(M0.cuda(), phi0.cuda())
    s.step(6)
    got_M = s.moments()
    got_phi = s.phi()
    want_M, want_phi = phase.run(LAT[lattice], M0, phi0, 6, TC["tau_l"], TC["tau_h"], TC["sigma"], TC["width"],
                                 TC["diffusivity"], body=(1e-6, 0.0, 0.0))
    err = group_errors(got_M, want_M)
    assert max(err.values()) < TOL[storage], err
    assert rel_max(got_phi, want_phi) < TOL[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_two_component_conserves_each_phase(storage):
    shape = (24, 24, 24)
    phi0 = synth.droplet(shape, 6.0, 4.0)
    M0 = torch.zeros((10,) + shape, dtype=torch.float64)
    s = Solver(shape, lattice=19, storage=storage, two_component=dict(TC, tau_h=1.0))
    s.set_moments(M0.cuda(), phi0.cuda())
    r0 = s.reduce()
    s.step(50)
    r1 = s.reduce()
    n = phi0.numel()
    tol = 1e-12 if storage == "f64" else 1e-6
    assert abs(r1[4] - r0[4]) < tol * r0[4]          # heavy phase: sum phi
    assert abs((n - r1[4]) - (n - r0[4])) < tol * n   # light phase: sum (1 - phi)
    assert abs(r1[0] - r0[0]) < tol * 1e-3 * n        # sum p*
