"""FP64 reductions and the closed-form solutions the oracle is checked against.

TEST INFRASTRUCTURE (oracle).

* reductions: sum p*, sum u (3), sum phi over fluid sites and E = <u.u>/2 over fluid sites
  (the kinetic-energy diagnostic of the Taylor-Green test, Sec. 3).
* Taylor-Green: E(t)/E(0) = exp(-6 nu k^2 t), k = 2 pi / N (Sec. 3).
* plane Poiseuille between halfway bounce-back walls (channel width H, walls midway between the
  last fluid and first solid node): steady u = g/(2 nu) eta (H - eta), and the start-up solution
  from rest as its Fourier sine series.
* Laplace law for a sphere, Delta P = 2 sigma / R (Sec. 3); for a cylinder, sigma / R.
"""
import math

import torch

from .lattice import CS2


def reductions(M, solid=None, phi=None):
    """[sum p*, sum ux, sum uy, sum uz, sum phi, E] over fluid sites, FP64."""
    M = torch.as_tensor(M, dtype=torch.float64)
    fluid = torch.ones(M.shape[1:], dtype=torch.bool)
    if solid is not None:
        fluid = ~torch.as_tensor(solid, dtype=torch.bool)
    n = fluid.sum()
    out = torch.zeros(6, dtype=torch.float64)
    out[0] = M[0][fluid].sum()
    for a in range(3):
        out[1 + a] = M[1 + a][fluid].sum()
    if phi is not None:
        out[4] = torch.as_tensor(phi, dtype=torch.float64)[fluid].sum()
    uu = (M[1:4] ** 2).sum(0)
    out[5] = 0.5 * uu[fluid].sum() / n
    return out


def kinetic_energy(M, solid=None):
    return float(reductions(M, solid)[5])


def taylor_green_energy_ratio(nu, n, t):
    k = 2.0 * math.pi / n
    return math.exp(-6.0 * nu * k * k * t)


def fit_decay_rate(times, values):
    """Least-squares slope of log(values) against times (a straight-line fit)."""
    t = torch.as_tensor(times, dtype=torch.float64)
    y = torch.log(torch.as_tensor(values, dtype=torch.float64))
    tm, ym = t.mean(), y.mean()
    return float(((t - tm) * (y - ym)).sum() / ((t - tm) ** 2).sum())


def poiseuille_steady(g, nu, H, eta):
    """u(eta) = g/(2 nu) eta (H - eta), eta the distance from the wall plane."""
    eta = torch.as_tensor(eta, dtype=torch.float64)
    return g / (2.0 * nu) * eta * (H - eta)


def poiseuille_startup(g, nu, H, eta, t, terms=2001):
    """Flow from rest under a constant acceleration g between no-slip walls:
    u = g/(2nu) eta (H - eta) - sum_{n odd} 4 g H^2 / (nu pi^3 n^3) sin(n pi eta / H) exp(-n^2 pi^2 nu t / H^2)."""
    eta = torch.as_tensor(eta, dtype=torch.float64)
    u = poiseuille_steady(g, nu, H, eta)
    for n in range(1, terms + 1, 2):
        amp = 4.0 * g * H * H / (nu * math.pi ** 3 * n ** 3)
        decay = math.exp(-(n * math.pi) ** 2 * nu * t / (H * H))
        if decay * amp < 1e-30:
            break
        u = u - amp * torch.sin(n * math.pi * eta / H) * decay
    return u


def laplace_pressure_jump(sigma, R, dim=3):
    return (2.0 if dim == 3 else 1.0) * sigma / R


def pressure(p_star, rho=1.0):
    """p = rho cs2 p* (definition of p* in Sec. 2)."""
    return rho * CS2 * torch.as_tensor(p_star, dtype=torch.float64)
