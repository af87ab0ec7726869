"""Pin of the pressure force of the two-component oracle (Sec. 2, force split: F_p = -p* cs2 grad rho).

The LB step evolves the rescaled pressure p* = p / (rho cs2) and works per unit mass, so its
pressure term is -cs2 grad p*. The physical term is -grad p / rho = -cs2 grad p* - cs2 p* grad rho
/ rho: F_p restores the second part. A fluid at rest at one uniform physical pressure p0 across a
density interface is then in mechanical equilibrium, although p* = p0 / (rho cs2) jumps across the
interface. Without F_p (or with a wrong sign or factor) the jump of p* is an unbalanced pressure
step, which launches sound waves of velocity amplitude about cs |p*_L - p*_H| / 2.

Case: a periodic column along x with a flat slab of the heavy phase (tanh profiles of width W),
rho_L = 0.5, rho_H = 1.5, equal viscosities, sigma = 0 (no capillary force), u = 0, p0 = 0.01.
The oracle must keep |u| below 1% of that acoustic scale, and the residual (the mismatch between
the lattice's own pressure gradient and the central-difference gradient of rho) must shrink when
the column, the interface and the time are refined together.
"""
import math

import torch

import oracle
from oracle import phase
from oracle.lattice import CS2

RHO_L, RHO_H, P0, TAU = 0.5, 1.5, 0.01, 0.8


def acoustic_scale(p0=P0):
    """cs |p*_L - p*_H| / 2: the velocity of the sound waves an unbalanced jump of p* launches."""
    return math.sqrt(CS2) * abs(p0 / (RHO_L * CS2) - p0 / (RHO_H * CS2)) / 2


def rest_slab_velocity(n=48, W=8.0, steps=60, p0=P0):
    """max |u| after `steps` two-component oracle steps from rest at uniform physical pressure p0."""
    x = torch.arange(n, dtype=torch.float64)
    phi = (0.5 * (torch.tanh(2 * (x - n / 4) / W) - torch.tanh(2 * (x - 3 * n / 4) / W))).reshape(1, 1, n)
    rho = RHO_L + phi * (RHO_H - RHO_L)
    M0 = torch.zeros((10, 1, 1, n), dtype=torch.float64)
    M0[0] = p0 / (rho * CS2)
    M, _ = phase.run(oracle.D3Q19, M0, phi, steps, TAU, TAU, 0.0, W, 0.1, rho_l=RHO_L, rho_h=RHO_H)
    return float(M[1:4].abs().max())


def pressure_pin_holds():
    return rest_slab_velocity() < 1e-2 * acoustic_scale()


def test_uniform_pressure_across_a_density_interface_stays_at_rest():
    u = rest_slab_velocity()
    assert u < 1e-2 * acoustic_scale(), (u, acoustic_scale())


def test_rest_residual_shrinks_under_refinement():
    coarse = rest_slab_velocity(48, 8.0, 60)
    fine = rest_slab_velocity(96, 16.0, 120)
    assert fine < 0.5 * coarse, (coarse, fine)


def test_rest_residual_is_driven_by_the_pressure():
    """At p0 = 0 p* is zero everywhere and F_p vanishes: the column stays exactly at rest."""
    assert rest_slab_velocity(p0=0.0) == 0.0
