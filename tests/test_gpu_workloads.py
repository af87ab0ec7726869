"""Workload-level checks on the GPU, one per measured configuration, against what the paper and the
mathematics fix: the Taylor-Green energy decay (Sec. 4) with exact conservation, the accuracy of
16-bit deviation storage against the FP64 path, and the Laplace law of a static droplet with the
conservation of each component. The FP64 GPU path stands in for the FP64 oracle where the oracle
cannot run the full workload; it is itself held to the oracle at 1e-12 (test_gpu_step.py and the
first test below)."""
import math

import pytest
import torch

import oracle
import synth
from oracle import diagnostics as dg
from oracle import lbm

from paper_2609_09160_gb300 import Solver

from _helpers import group_errors

pytestmark = pytest.mark.gpu


def test_taylor_green_32_fp64_decay_conservation_and_oracle():
    """D3Q19, FP64 storage, 32^3 periodic Taylor-Green (U0 = 0.02, k = 2 pi/32), tau = 0.8, 100
    steps: E/E0 = exp(-6 nu k^2 t) with nu = (tau - 1/2)/3 (Sec. 4) within 1e-2, the fitted
    viscosity within 1e-2, mass and momentum conserved to round-off, and the final state equal to
    the oracle's 100-step run within 1e-12."""
    n, tau, steps, every = 32, 0.8, 100, 5
    M0 = synth.taylor_green(n, 0.02, tau)
    s = Solver((n, n, n), lattice=19, tau=tau, storage="f64")
    s.set_moments(M0.cuda())
    r0 = s.reduce()
    ts, es = [0], [dg.kinetic_energy(M0)]
    for t in range(every, steps + 1, every):
        s.step(every)
        ts.append(t)
        es.append(dg.kinetic_energy(s.moments().cpu()))
    r1 = s.reduce()
    nu = lbm.viscosity(tau)
    k = 2 * math.pi / n
    nu_fit = -dg.fit_decay_rate(ts, es) / (6 * k * k)
    assert abs(nu_fit - nu) / nu < 1e-2
    ratio = es[-1] / es[0]
    assert abs(ratio - dg.taylor_green_energy_ratio(nu, n, steps)) < 1e-2 * ratio
    scale_p, scale_u = float(M0[0].abs().sum()), float(M0[1:4].abs().sum())
    assert abs(r1[0] - r0[0]) < 1e-13 * scale_p
    for a in (1, 2, 3):
        assert abs(r1[a] - r0[a]) < 1e-13 * scale_u
    want = lbm.run(oracle.D3Q19, M0, steps, tau)
    err = group_errors(s.moments().cpu(), want)
    assert max(err.values()) < 1e-12, err


def _velocity_errors(M, ref):
    du = M[1:4] - ref[1:4]
    return (float(torch.linalg.norm(du) / torch.linalg.norm(ref[1:4])),
            float(du.abs().max() / ref[1:4].abs().max()))


def test_16bit_deviation_storage_d3q27_taylor_green_64():
    """D3Q27, 64^3 periodic Taylor-Green (U0 = 0.04) plus a random-phase perturbation of RMS 0.01,
    tau = 0.55, 500 steps, every storage dtype against FP64 storage on the same GPU. Velocity
    error, relative in the L2 norm over the box: FP32 < 1e-5, FP16 < 1e-3 (measured 5.8e-4 with
    the default stochastic rounding, 4.8e-4 with round-to-nearest; in the max norm over sites FP16
    reaches ~2e-3, bounded here by 5e-3), BF16 < 1e-2 (measured 4.7e-3; 8 significand bits)."""
    n, tau, steps = 64, 0.55, 500
    M0 = synth.taylor_green_perturbed(n, 0.04, tau, 0.01, seed=3, dtype=torch.float64, device="cuda")
    out = {}
    for key, st, rounding in (("f64", "f64", "stochastic"), ("f32", "f32", "stochastic"), ("f16", "f16", "stochastic"),
                              ("bf16", "bf16", "stochastic"), ("f16rn", "f16", "nearest")):
        s = Solver((n, n, n), lattice=27, tau=tau, storage=st, rounding=rounding)
        s.set_moments(M0 if st == "f64" else M0.float())
        s.step(steps)
        out[key] = s.moments()
        del s
    ref = out["f64"]
    l2, mx = _velocity_errors(out["f32"], ref)
    assert l2 < 1e-5 and mx < 1e-5, (l2, mx)
    l2, mx = _velocity_errors(out["f16"], ref)
    assert l2 < 1e-3 and mx < 5e-3, (l2, mx)
    l2, mx = _velocity_errors(out["bf16"], ref)
    assert l2 < 1e-2, (l2, mx)
    l2, mx = _velocity_errors(out["f16rn"], ref)
    assert l2 < 1e-3 and mx < 5e-3, (l2, mx)


@pytest.mark.slow
def test_16bit_deviation_storage_d3q27_taylor_green_512_crop():
    """The full-size configuration: D3Q27, 512^3 Taylor-Green + perturbation, tau = 0.55, 500
    steps, errors of FP32 and FP16 storage against FP64 storage on a 64^3 crop. With the default
    stochastic rounding FP16 stays below 1e-3 (measured 5.9e-4); round-to-nearest (the survey's
    reading, LBF_ROUND_NEAREST) lets the slowly evolving flow freeze and exceeds 2e-3 (measured
    8.0e-3), which this test also pins so that a silent loss of the stochastic path shows."""
    n, tau, steps = 512, 0.55, 500
    crop = (slice(None), slice(0, 64), slice(0, 64), slice(0, 64))
    M0 = synth.taylor_green_perturbed(n, 0.04, tau, 0.01, seed=3, dtype=torch.float32, device="cuda")
    out = {}
    for key, st, rounding in (("f64", "f64", "stochastic"), ("f32", "f32", "stochastic"),
                              ("f16", "f16", "stochastic"), ("f16rn", "f16", "nearest")):
        s = Solver((n, n, n), lattice=27, tau=tau, storage=st, rounding=rounding)
        s.set_moments(M0)
        s.step(steps)
        out[key] = s.moments()[crop].clone()
        del s
        torch.cuda.empty_cache()
    ref = out["f64"]
    l2, mx = _velocity_errors(out["f32"], ref)
    assert l2 < 1e-5 and mx < 1e-5, (l2, mx)
    l2, mx = _velocity_errors(out["f16"], ref)
    assert l2 < 1e-3 and mx < 5e-3, (l2, mx)
    l2_rn, _ = _velocity_errors(out["f16rn"], ref)
    assert l2_rn > 2e-3, l2_rn


def test_droplet_128_laplace_law_and_conservation():
    """Two-component D3Q19 FP32, 128^3 periodic static droplet, R = 20, W = 4, sigma = 0.03,
    D = 0.1, equal densities, tau = 1 in both phases, 5000 steps: the pressure jump
    p = rho cs2 p* inside minus outside gives sigma = dp R / 2 within 10% (Laplace law in 3-D; the
    paper's own droplet gives sigma 6.8% low, Sec. 4), sum(phi) and sum(p*) are conserved and the
    spurious currents stay small."""
    n, R, W, sigma = 128, 20.0, 4.0, 0.03
    shape = (n, n, n)
    s = Solver(shape, lattice=19, storage="f32",
               two_component=dict(rho_l=1.0, rho_h=1.0, tau_l=1.0, tau_h=1.0, sigma=sigma, width=W, diffusivity=0.1))
    phi0 = synth.droplet(shape, R, W, dtype=torch.float32, device="cuda")
    s.set_moments(torch.zeros((10,) + shape, dtype=torch.float32, device="cuda"), phi0)
    r0 = s.reduce()
    s.step(5000)
    r1 = s.reduce()
    M, phi = s.moments(), s.phi()
    x = torch.arange(n, dtype=torch.float64, device=M.device)
    zz, yy, xx = torch.meshgrid(x, x, x, indexing="ij")
    r = torch.sqrt((xx - n / 2) ** 2 + (yy - n / 2) ** 2 + (zz - n / 2) ** 2)
    r_eff = (3.0 * float(phi.sum()) / (4.0 * math.pi)) ** (1.0 / 3.0)
    p = dg.pressure(M[0].cpu()).to(M.device)
    dp = float(p[r < r_eff - 2 * W].mean() - p[r > r_eff + 2 * W].mean())
    assert abs(dp - dg.laplace_pressure_jump(sigma, r_eff)) < 0.10 * dg.laplace_pressure_jump(sigma, r_eff)
    assert abs(r1[4] - r0[4]) < 1e-6 * r0[4]
    assert abs(r1[0] - r0[0]) < 1e-5 * float(M[0].abs().sum())
    assert float(M[1:4].abs().max()) < 1e-4
