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


# density and viscosity contrast (Sec. 2 force split F = F^s + F^b + F^p + F^nu), with walls and a
# body acceleration: the pressure force needs p* != 0, so the state carries a uniform offset
TCC = dict(rho_l=0.5, rho_h=1.5, tau_l=0.8, tau_h=1.1, sigma=0.02, width=4.0, diffusivity=0.1,
           body_accel=(0.0, 2e-6, -1e-6))


@pytest.mark.parametrize("lattice", [19, 27, 127])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("walls", [False, True])
def test_density_contrast_matches_oracle(lattice, storage, walls):
    shape = (12, 15, 33)
    phi0 = synth.droplet(shape, 5.0, 4.0)
    M0 = synth.random_moments(shape, seed=81, p_scale=1e-3, u_scale=2e-3, neq_scale=1e-5)
    M0[0] += 0.03
    mask = synth.channel_walls(shape) if walls else None
    s = Solver(shape, lattice=lattice, storage=storage, two_component=TCC, force=(1e-6, 0.0, 0.0), mask=mask)
    s.set_moments(M0.cuda(), phi0.cuda())
    s.step(6)
    got_M = s.moments()
    got_phi = s.phi()
    want_M, want_phi = phase.run(LAT[lattice], M0, phi0, 6, TCC["tau_l"], TCC["tau_h"], TCC["sigma"], TCC["width"],
                                 TCC["diffusivity"], rho_l=TCC["rho_l"], rho_h=TCC["rho_h"], body=(1e-6, 0.0, 0.0),
                                 solid=mask, body_accel=TCC["body_accel"])
    err = group_errors(got_M, want_M)
    assert max(err.values()) < TOL[storage], err
    assert rel_max(got_phi, want_phi) < TOL[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_layered_poiseuille_on_the_gpu(storage):
    """The layered two-phase Poiseuille flow of Sec. 4 (light phase rho 0.5 against one wall, heavy
    phase rho 1.5 with 8x the viscosity against the other, body acceleration along the layers):
    started on the continuum steady state of the diffuse-interface model, 600 GPU steps keep the
    profile within 1% of it, as the oracle does."""
    from test_oracle_layered import A_Z, H, NU1, NU2, RHO1, RHO2, W, diffuse_steady
    from oracle.lattice import CS2

    nx = H + 2
    shape = (1, 1, nx)
    xi = torch.arange(nx, dtype=torch.float64) - 0.5
    phi0 = (0.5 * (1 + torch.tanh(2 * (xi - H / 2) / W))).reshape(shape).clone()
    phi0[..., 0], phi0[..., -1] = 0.0, 1.0
    solid = torch.zeros(shape, dtype=torch.bool)
    solid[..., 0] = solid[..., -1] = True
    want = diffuse_steady(H, W, NU1, NU2, RHO1, RHO2, A_Z, xi[1:-1])
    M0 = torch.zeros((10,) + shape, dtype=torch.float64)
    M0[3, 0, 0, 1:-1] = want
    M0[6] = M0[3] * M0[3]
    tc = dict(rho_l=RHO1, rho_h=RHO2, tau_l=NU1 / CS2 + 0.5, tau_h=NU2 / CS2 + 0.5, sigma=0.03, width=W,
              diffusivity=0.1, body_accel=(0.0, 0.0, A_Z))
    s = Solver(shape, lattice=19, storage=storage, two_component=tc, mask=solid)
    s.set_moments(M0.cuda(), phi0.cuda())
    s.step(600)
    got = s.moments()[3, 0, 0, 1:-1].cpu()
    dev = float((got - want).abs().max() / want.abs().max())
    assert dev < 1e-2, dev
