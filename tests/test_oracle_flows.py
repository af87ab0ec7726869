"""Pins of the oracle against closed-form flow solutions and the paper's printed values:
shear-wave viscosity, Taylor-Green energy decay (Sec. 4, Eq. tg), steady and start-up plane
Poiseuille flow between halfway bounce-back walls, and the memory-footprint model of Sec. 3."""
import json
import math
import os

import pytest
import torch

import oracle
import synth
from oracle import diagnostics as dg
from oracle import lbm

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
LATS = [oracle.D3Q19, oracle.D3Q27]
ids = lambda l: l.name  # noqa: E731


def shear_wave_viscosity(lat, N, tau, steps):
    """Decay rate of u_x = U sin(2 pi y / N) (an exact Navier-Stokes mode): nu k^2."""
    y = torch.arange(N, dtype=torch.float64).reshape(1, N, 1)
    mode = torch.sin(2 * math.pi * y / N)
    u = torch.zeros((3, 1, N, 1), dtype=torch.float64)
    u[0] = 1e-3 * mode
    M0 = synth.moments_from_velocity(torch.zeros((1, N, 1), dtype=torch.float64), u, tau)
    ts, amps = [], []
    lbm.run(lat, M0, steps, tau,
            callback=lambda t, M: (ts.append(t), amps.append(float((M[1] * mode).sum()) * 2 / N)))
    k = 2 * math.pi / N
    return -dg.fit_decay_rate(ts, amps) / (k * k)


@pytest.mark.parametrize("lat", LATS, ids=ids)
@pytest.mark.parametrize("tau", [0.55, 0.8, 1.4])
def test_shear_wave_viscosity(lat, tau):
    """nu = cs2 (tau - 1/2) (text under Eq. pullLB), measured on a pure shear mode."""
    nu = lbm.viscosity(tau)
    nu_fit = shear_wave_viscosity(lat, 64, tau, 120)
    assert abs(nu_fit - nu) / nu < 2e-3


def taylor_green_fit(lat, n, u0, tau, steps, every=5):
    M0 = synth.taylor_green(n, u0, tau)
    ts, es = [0], [dg.kinetic_energy(M0)]
    sums0 = dg.reductions(M0)
    last = {}

    def cb(t, M):
        last["M"] = M
        if t % every == 0:
            ts.append(t)
            es.append(dg.kinetic_energy(M))
    lbm.run(lat, M0, steps, tau, callback=cb)
    k = 2 * math.pi / n
    nu_fit = -dg.fit_decay_rate(ts, es) / (6 * k * k)
    return nu_fit, es, ts, sums0, dg.reductions(last["M"])


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_taylor_green_decay_config_32(lat):
    """32^3 periodic Taylor-Green, U0 = 0.02, tau = 0.8 (nu = 0.1), 100 steps: the energy follows
    E/E0 = exp(-6 nu k^2 t) (Sec. 4) and mass and momentum are exactly conserved."""
    nu = lbm.viscosity(0.8)
    nu_fit, es, ts, s0, s1 = taylor_green_fit(lat, 32, 0.02, 0.8, 100)
    assert abs(nu_fit - nu) / nu < 1e-2
    ratio = es[-1] / es[0]
    assert abs(ratio - dg.taylor_green_energy_ratio(nu, 32, ts[-1])) < 1e-2 * ratio
    M0 = synth.taylor_green(32, 0.02, 0.8)
    scale = float(M0[0].abs().sum()), float(M0[1:4].abs().sum())
    assert abs(float(s1[0] - s0[0])) < 1e-13 * scale[0]
    assert (s1[1:4] - s0[1:4]).abs().max() < 1e-13 * scale[1]


def test_taylor_green_with_the_papers_parameters():
    """The paper's TG parameters (nu = 0.04074, U0 = 0.04; Sec. 4) on a 32^3 box: the fitted
    viscosity, fitted over the initial decay range, matches the input within 1e-2 (the paper
    reports ~1.3e-3 at 512^3, where the Reynolds number is 80 instead of 5)."""
    g = GOLDEN["taylor_green"]
    for v in g["nu_fit"].values():
        assert abs(v - g["nu"]) / g["nu"] < 2e-3
    tau = 3 * g["nu"] + 0.5
    nu_fit, *_ = taylor_green_fit(oracle.D3Q19, 32, g["U0"], tau, 40, every=4)
    assert abs(nu_fit - g["nu"]) / g["nu"] < 1e-2


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_poiseuille_steady_profile(lat):
    """Walls on y = 0 and y = ny-1, H = ny - 2 fluid rows, walls midway: the steady profile is the
    parabola g/(2 nu) eta (H - eta), eta = y - 1/2."""
    H, tau, g = 16, 0.9, 1e-5
    ny = H + 2
    M0, solid = synth.channel((1, ny, 1), 0.0, seed=0)
    M = lbm.run(lat, M0, 2500, tau, force=(g, 0.0, 0.0), solid=solid)
    eta = torch.arange(ny, dtype=torch.float64) - 0.5
    want = dg.poiseuille_steady(g, lbm.viscosity(tau), H, eta)[1:-1]
    got = M[1, 0, 1:-1, 0]
    assert float((got - want).abs().max() / want.max()) < 1e-2
    assert M[2:4].abs().max() < 1e-18


def test_poiseuille_startup_series():
    """Start-up from rest (the channel configuration at reduced width): the velocity profile
    follows the sine-series solution of the unsteady Stokes problem."""
    H, tau, g, steps = 30, 0.9, 1e-6, 600
    ny = H + 2
    M0, solid = synth.channel((2, ny, 3), 0.0, seed=0)
    M = lbm.run(oracle.D3Q19, M0, steps, tau, force=(g, 0.0, 0.0), solid=solid)
    eta = torch.arange(ny, dtype=torch.float64) - 0.5
    want = dg.poiseuille_startup(g, lbm.viscosity(tau), H, eta, steps)[1:-1]
    got = M[1, :, 1:-1, :].mean(dim=(0, 2))
    assert float(torch.linalg.norm(got - want) / torch.linalg.norm(want)) < 1e-2


def test_memory_footprint_model():
    """Sec. 3: M = N n_fields b gives 20/38/54 GB (FP64) and 10/19/27 GB (FP32) at 512^3,
    with GB = 2^30 bytes, and the quoted percentage reductions."""
    g = GOLDEN["memory_512"]
    N = g["sites"]
    assert N == 512 ** 3
    for key, nf in g["fields"].items():
        assert N * nf * 8 == g["GB_fp64"][key] * 2 ** 30
        assert N * nf * 4 == g["GB_fp32"][key] * 2 ** 30
    for lat, nf in (("D3Q19", 38), ("D3Q27", 54)):
        assert abs(100 * (1 - 20 / nf) - g["reduction_percent"][lat]) < 0.05
