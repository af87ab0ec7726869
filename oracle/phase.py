"""FP64 reference of the two-component coupling: conservative Allen-Cahn phase field (FTCS) and
the capillary force, Eq. (ACeq) and the force split of Sec. 2.

TEST INFRASTRUCTURE (oracle).

* Density and viscosity blending: rho(phi) = rho_L + phi (rho_H - rho_L),
  nu(phi) = nu_L + phi (nu_H - nu_L), phi = 1 heavy, phi = 0 light; omega = 1/(nu/cs2 + 1/2).
* Lattice stencils with D3Q27 weights (end of Sec. 2):
    gradient   d_a psi = (1/cs2) sum_i w_i psi(x + c_i) c_ia            (as printed)
    Laplacian  lap psi = (2/cs2) sum_i w_i (psi(x + c_i) - psi(x))       (the printed form is
               garbled; this is the isotropic second-order form that the printed one reduces to)
    divergence div V   = (1/cs2) sum_i w_i c_i . V(x + c_i)              (gradient stencil applied
               to each component)
* Allen-Cahn by FTCS in flux form: phi' = phi - div(phi u) + D lap phi - lambda div(phi(1-phi) n),
  lambda = 4 D / W, n = grad phi / max(|grad phi|, 1e-12). The flux form is identical to the printed
  advective form for a divergence-free u and keeps sum(phi) exact on a periodic box.
* Chemical potential mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap phi, beta = 12 sigma / W,
  kappa = 3 sigma W / 2; capillary force F_s = mu grad phi.
* Density contrast (Sec. 2, force split F = F_s + F_b + F_p + F_nu):
    F_p  = -p* cs2 grad rho                                          (as printed)
    F_nu = nu S . grad rho,  S = -(omega / cs2) a*_neq               (reading: the printed
           coefficient "nu omega cs2 a*_neq" is dimensionally garbled; this is the viscous stress
           nu (grad u + grad u^T) . grad rho that the per-unit-mass LB step leaves out, with the
           Chapman-Enskog strain rate of the raw, uncorrected second moments a*_neq = a*2 - a*1 a*1)
  Both vanish when rho_L = rho_H. F_b may be given as a body acceleration a (F_b = rho(phi) a).
* Walls (solid mask): halfway bounce-back for the populations; the phase field is not advanced at
  solid sites (they keep their phi, u = 0 there), so a wall in contact with a single bulk phase
  exchanges no phi. Wetting (a contact line on a wall) is not modelled.
"""
import torch

from . import lbm
from .lattice import CS2, D3Q27


def shift_to(x, c):
    """Value of field x at site (position + c), periodic."""
    return torch.roll(x, shifts=(-int(c[2]), -int(c[1]), -int(c[0])), dims=(-3, -2, -1))


def gradient(psi):
    g = torch.zeros((3,) + tuple(psi.shape), dtype=torch.float64)
    for i in range(D3Q27.Q):
        ci = D3Q27.ci[i]
        nb = shift_to(psi, ci)
        for a in range(3):
            if ci[a] != 0:
                g[a] += D3Q27.w[i] * float(ci[a]) * nb
    return g / CS2


def laplacian(psi):
    acc = torch.zeros_like(psi)
    for i in range(D3Q27.Q):
        acc += D3Q27.w[i] * (shift_to(psi, D3Q27.ci[i]) - psi)
    return 2.0 * acc / CS2


def divergence(V):
    acc = torch.zeros(V.shape[1:], dtype=torch.float64)
    for i in range(D3Q27.Q):
        ci = D3Q27.ci[i]
        for a in range(3):
            if ci[a] != 0:
                acc += D3Q27.w[i] * float(ci[a]) * shift_to(V[a], ci)
    return acc / CS2


def normal(phi):
    g = gradient(phi)
    mag = torch.sqrt((g * g).sum(0))
    return g / torch.clamp(mag, min=1e-12)


def allen_cahn_step(phi, u, D, W):
    lam = 4.0 * D / W
    return (phi - divergence(phi.unsqueeze(0) * u) + D * laplacian(phi)
            - lam * divergence((phi * (1.0 - phi)).unsqueeze(0) * normal(phi)))


def chemical_potential(phi, sigma, W):
    beta = 12.0 * sigma / W
    kappa = 1.5 * sigma * W
    return 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kappa * laplacian(phi)


def capillary_force(phi, sigma, W):
    return chemical_potential(phi, sigma, W).unsqueeze(0) * gradient(phi)


def density(phi, rho_l, rho_h):
    return rho_l + phi * (rho_h - rho_l)


def omega(phi, tau_l, tau_h):
    nu_l, nu_h = CS2 * (tau_l - 0.5), CS2 * (tau_h - 0.5)
    nu = nu_l + phi * (nu_h - nu_l)
    return 1.0 / (nu / CS2 + 0.5)


def pressure_force(phi, p, rho_l, rho_h):
    """F_p = -p* cs2 grad rho, grad rho = (rho_H - rho_L) grad phi (Sec. 2)."""
    return -(CS2 * p).unsqueeze(0) * ((rho_h - rho_l) * gradient(phi))


def viscous_force(phi, a2neq, tau_l, tau_h, rho_l, rho_h):
    """F_nu_a = nu S_ab d_b rho with S = -(omega / cs2) a*_neq (reading of Sec. 2, see header)."""
    nu = CS2 * (tau_l - 0.5) + phi * (CS2 * (tau_h - tau_l))
    coef = -(nu * omega(phi, tau_l, tau_h) / CS2)
    grho = (rho_h - rho_l) * gradient(phi)
    return coef.unsqueeze(0) * torch.einsum("ab...,b...->a...", a2neq, grho)


def total_force(phi, p, body, sigma, W, a2neq=None, rho_l=1.0, rho_h=1.0, tau_l=1.0, tau_h=1.0,
                body_accel=None):
    """F = F_s + F_b + F_p + F_nu (F_p and F_nu only with a density contrast). body is a force per
    unit volume; body_accel, if given, adds rho(phi) a."""
    F = capillary_force(phi, sigma, W) + lbm.as_field(body, phi.shape)
    if body_accel is not None:
        F = F + density(phi, rho_l, rho_h).unsqueeze(0) * lbm.as_field(body_accel, phi.shape)
    if rho_l != rho_h:
        F = F + pressure_force(phi, p, rho_l, rho_h) + viscous_force(phi, a2neq, tau_l, tau_h, rho_l, rho_h)
    return F


def run(lat, M0, phi0, steps, tau_l, tau_h, sigma, W, D, rho_l=1.0, rho_h=1.0,
        body=(0.0, 0.0, 0.0), callback=None, solid=None, body_accel=None):
    """Two-component run. State (populations f, phi). Order of one step:
    phi^{n+1} = AC(phi^n, u^n); collide with F^n, rho(phi^n), omega(phi^n) and stream;
    F^{n+1} = F(phi^{n+1}, p*^{n+1}, a*_neq^{n+1}) is the force of the new state (Eq. corr at t+1),
    with p* and a*_neq taken from the raw moments of the streamed populations. F^0 uses the
    non-equilibrium part N = A - u u of the initial state.
    solid: bool (nz, ny, nx) or None (see the header for walls). Solid sites keep M0 and phi0.
    Returns (M, phi) after `steps` steps; callback(t, M, phi) after each step."""
    M0 = torch.as_tensor(M0, dtype=torch.float64)
    phi = torch.as_tensor(phi0, dtype=torch.float64).clone()
    shape = phi.shape
    if solid is not None:
        solid = torch.as_tensor(solid, dtype=torch.bool)
    kw = dict(rho_l=rho_l, rho_h=rho_h, tau_l=tau_l, tau_h=tau_h, body_accel=body_accel)
    p0, u0, A0 = lbm.unpack(M0)
    N0 = A0 - torch.einsum("a...,b...->ab...", u0, u0)
    F = total_force(phi, p0, body, sigma, W, a2neq=N0, **kw)
    rho = density(phi, rho_l, rho_h)
    f = lbm.populations_from_moments(lat, M0, F, rho)
    M = M0
    for t in range(1, steps + 1):
        rho = density(phi, rho_l, rho_h)
        om = omega(phi, tau_l, tau_h)
        _, u, _ = lbm.macroscopic(lat, f, F, rho)
        if solid is not None:
            u = torch.where(solid.unsqueeze(0), torch.zeros_like(u), u)
        phi_new = allen_cahn_step(phi, u, D, W)
        if solid is not None:
            phi_new = torch.where(solid, phi, phi_new)
        f = lbm.step(lat, f, F, rho, om, solid)
        phi = phi_new
        a0, a1, a2 = lbm.hermite_project(lat, f)
        F = total_force(phi, a0, body, sigma, W, a2neq=a2 - torch.einsum("a...,b...->ab...", a1, a1), **kw)
        if callback is not None or t == steps:
            M = lbm.moments_from_populations(lat, f, F, density(phi, rho_l, rho_h))
            if solid is not None:
                M = torch.where(solid.unsqueeze(0), M0, M)
            if callback is not None:
                callback(t, M, phi)
    return M, phi
