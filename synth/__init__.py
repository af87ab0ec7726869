"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This package only builds initial states and parameter fields; it holds none of the stepping
arithmetic. Every generator is deterministic for a given seed (numpy PCG64 for random draws,
closed-form trigonometric fields otherwise) and returns torch tensors on the requested device
and dtype, laid out as the public moment state (10, nz, ny, nx):
[p*, ux, uy, uz, Axx, Ayy, Azz, Axy, Axz, Ayz], with A the total second Hermite coefficient.

Initial second moments follow the paper's velocity form (Sec. 2): A = u u + a_neq with either
a_neq = 0 (equilibrium start) or the Chapman-Enskog value a_neq = -(cs2/omega)(du + du^T), whose
velocity gradients are taken spectrally (exact for the trigonometric fields generated here).
"""
import math

import numpy as np
import torch

CS2 = 1.0 / 3.0
SYM = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _pack(p, u, A):
    comps = [p, u[0], u[1], u[2]] + [A[a][b] for (a, b) in SYM]
    return torch.stack(comps, 0)


def _grid(n3, dtype, device):
    nz, ny, nx = n3
    z = torch.arange(nz, dtype=dtype, device=device).reshape(nz, 1, 1)
    y = torch.arange(ny, dtype=dtype, device=device).reshape(1, ny, 1)
    x = torch.arange(nx, dtype=dtype, device=device).reshape(1, 1, nx)
    return x, y, z


def spectral_gradient(u):
    """G[a, b] = d u_a / d x_b on a periodic grid (axes z, y, x), exact for trigonometric fields
    below the Nyquist wave number."""
    nz, ny, nx = u.shape[1:]
    dev = u.device

    def wavenumbers(n, view):
        k = torch.fft.fftfreq(n, d=1.0, device=dev).to(u.dtype) * (2 * math.pi)
        if n % 2 == 0:
            k[n // 2] = 0.0  # keep derivatives of real fields real
        return k.reshape(view)

    ks = (wavenumbers(nx, (1, 1, nx)), wavenumbers(ny, (1, ny, 1)), wavenumbers(nz, (nz, 1, 1)))
    G = torch.empty((3, 3) + tuple(u.shape[1:]), dtype=u.dtype, device=dev)
    for a in range(3):
        U = torch.fft.fftn(u[a], dim=(0, 1, 2))
        for b in range(3):
            G[a, b] = torch.fft.ifftn(1j * ks[b] * U, dim=(0, 1, 2)).real
    return G


def moments_from_velocity(p, u, tau=None, chapman_enskog=True):
    """Public moment state from p*, u; A = u u (+ Chapman-Enskog a_neq when tau is given)."""
    A = [[u[a] * u[b] for b in range(3)] for a in range(3)]
    if chapman_enskog and tau is not None:
        G = spectral_gradient(u)
        omega = 1.0 / tau
        for a in range(3):
            for b in range(3):
                A[a][b] = A[a][b] - (CS2 / omega) * (G[a, b] + G[b, a])
    return _pack(p, u, A)


def taylor_green_velocity(shape, u0, dtype=torch.float64, device="cpu"):
    """Eq. (tg) velocity and pressure on a periodic box, coordinates 2 pi i / N (0-based)."""
    nz, ny, nx = shape
    x, y, z = _grid(shape, dtype, device)
    X, Y, Z = 2 * math.pi * x / nx, 2 * math.pi * y / ny, 2 * math.pi * z / nz
    ux = u0 * torch.sin(X) * torch.cos(Y) * torch.cos(Z)
    uy = -u0 * torch.cos(X) * torch.sin(Y) * torch.cos(Z)
    uz = torch.zeros_like(ux * uy)
    p = (u0 * u0 / 16.0) * (torch.cos(2 * X) + torch.cos(2 * Y)) * (2.0 + torch.cos(2 * Z))
    u = torch.stack([ux.expand(shape), uy.expand(shape), uz.expand(shape)], 0)
    return p.expand(shape).contiguous(), u.contiguous()


def taylor_green(n, u0, tau, chapman_enskog=True, dtype=torch.float64, device="cpu"):
    """Taylor-Green vortex of Sec. 3 on an n^3 periodic box with rho = 1: p* = p/(rho cs2)."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    p, u = taylor_green_velocity(shape, u0, dtype, device)
    return moments_from_velocity(p / CS2, u, tau, chapman_enskog)


def random_phase_perturbation(shape, amplitude, seed, n_modes=16, kmax=4, dtype=torch.float64,
                              device="cpu"):
    """Solenoidal perturbation: curl of a vector potential made of `n_modes` Fourier modes with
    integer wave vectors in [-kmax, kmax]^3 \\ {0} and random phases, scaled to RMS |du| = amplitude."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    x, y, z = _grid(shape, dtype, device)
    du = torch.zeros((3,) + tuple(shape), dtype=dtype, device=device)
    for _ in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(k != 0):
                break
        a = rng.standard_normal(3)
        phase = rng.uniform(0.0, 2 * math.pi)
        kv = (2 * math.pi * k[0] / nx, 2 * math.pi * k[1] / ny, 2 * math.pi * k[2] / nz)
        theta = kv[0] * x + kv[1] * y + kv[2] * z + phase
        s = -torch.sin(theta)
        # curl(a cos(theta)) = grad(cos theta) x a = -sin(theta) k x a
        kxa = (kv[1] * a[2] - kv[2] * a[1], kv[2] * a[0] - kv[0] * a[2], kv[0] * a[1] - kv[1] * a[0])
        for c in range(3):
            du[c] += float(kxa[c]) * s
    rms = torch.sqrt((du * du).sum(0).mean())
    return du * (amplitude / rms)


def taylor_green_perturbed(n, u0, tau, amplitude, seed, dtype=torch.float64, device="cpu"):
    """Taylor-Green plus a seeded random-phase solenoidal perturbation (Chapman-Enskog A)."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    p, u = taylor_green_velocity(shape, u0, dtype, device)
    u = u + random_phase_perturbation(shape, amplitude, seed, dtype=dtype, device=device)
    return moments_from_velocity(p / CS2, u, tau, True)


def channel_walls(shape, device="cpu"):
    """Solid mask (nz, ny, nx) with walls on the planes y = 0 and y = ny - 1."""
    nz, ny, nx = shape
    solid = torch.zeros(shape, dtype=torch.bool, device=device)
    solid[:, 0, :] = True
    solid[:, ny - 1, :] = True
    return solid


def channel(shape, noise, seed, dtype=torch.float64, device="cpu"):
    """Channel at rest: p* uniform in [-noise, noise] (rho = 1 +/- noise), u = 0, A = 0."""
    rng = np.random.default_rng(seed)
    M = torch.zeros((10,) + tuple(shape), dtype=dtype, device=device)
    M[0] = torch.from_numpy(rng.uniform(-noise, noise, size=shape)).to(dtype=dtype, device=device)
    return M, channel_walls(shape, device)


def droplet(shape, radius, width, dtype=torch.float64, device="cpu"):
    """phi = (1 + tanh(2 (R - r) / W)) / 2 centred at (N/2, N/2, N/2), heavy phase inside."""
    nz, ny, nx = shape
    x, y, z = _grid(shape, dtype, device)
    r = torch.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
    return (0.5 * (1.0 + torch.tanh(2.0 * (radius - r) / width))).expand(shape).contiguous()


def cylinder(shape, radius, width, dtype=torch.float64, device="cpu"):
    """Column along z: phi = (1 + tanh(2 (R - r) / W)) / 2 with r the distance from the z axis."""
    nz, ny, nx = shape
    x, y, z = _grid(shape, dtype, device)
    r = torch.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2)
    return (0.5 * (1.0 + torch.tanh(2.0 * (radius - r) / width))).expand(shape).contiguous()


def random_moments(shape, seed, p_scale=1e-3, u_scale=0.05, neq_scale=1e-3, dtype=torch.float64,
                   device="cpu"):
    """Random state that exercises every term: p* ~ U(-p, p), u ~ U(-u, u), A = u u + sym noise."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))

    def draw(scale):
        return torch.from_numpy(rng.uniform(-scale, scale, size=n).reshape(shape)).to(dtype=dtype,
                                                                                     device=device)

    p = draw(p_scale)
    u = torch.stack([draw(u_scale) for _ in range(3)], 0)
    A = [[None] * 3 for _ in range(3)]
    for (a, b) in SYM:
        A[a][b] = u[a] * u[b] + draw(neq_scale)
        A[b][a] = A[a][b]
    return _pack(p, u, A)


def random_field(shape, std, seed, dtype=torch.float64, device="cpu", mask=None):
    """(3, *shape) Gaussian field N(0, std^2), zero where `mask` (solid) is set."""
    rng = np.random.default_rng(seed)
    F = torch.from_numpy(rng.standard_normal((3,) + tuple(shape)) * std).to(dtype=dtype, device=device)
    if mask is not None:
        F = F * (~mask.to(device)).to(dtype).unsqueeze(0)
    return F


def random_mask(shape, fraction, seed, device="cpu"):
    """Scattered solid sites (a porous-medium-like mask) for bounce-back coverage."""
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.random(shape) < fraction).to(device)
