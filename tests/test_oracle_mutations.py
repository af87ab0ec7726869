"""Planted-mistake checks: each test swaps one oracle function for a copy with a plausible
mistake (a dropped term, a wrong sign, index or factor, a transposed operand) and asserts that
the oracle's pins notice it. All mutants live here, on the CPU; the oracle itself is untouched."""
import math

import pytest
import torch

import oracle
import synth
from oracle import diagnostics as dg
from oracle import lbm, moment_form, phase
from oracle.lattice import CS2


def pins_fail():
    """Run a battery of fast pins; return the names of the ones that fail."""
    failed = []
    lat = oracle.D3Q19
    # 1. literal moment form (its own arithmetic) vs the population form, with force and walls
    shape = (4, 4, 4)
    M = synth.random_moments(shape, seed=31)
    F = synth.random_field(shape, 1e-3, seed=32)
    solid = synth.random_mask(shape, 0.2, seed=33)
    a = lbm.step_moments(lat, M, 0.7, F, F, solid)
    b = torch.tensor(moment_form.step(lat, M.tolist(), 0.7, F.tolist(), F.tolist(), solid.tolist()),
                     dtype=torch.float64)
    if not float((a - b).abs().max() / b.abs().max()) < 1e-13:
        failed.append("literal")
    # 2. momentum grows by N F / rho per step
    M0 = synth.random_moments((3, 4, 5), seed=12)
    Fu = torch.tensor([1e-4, -2e-4, 3e-5], dtype=torch.float64)
    Mt = lbm.run(lat, M0, 3, 0.7, force=Fu)
    grow = Mt[1:4].sum((1, 2, 3)) - M0[1:4].sum((1, 2, 3))
    if not float((grow - 3 * 60 * Fu).abs().max()) < 1e-15:
        failed.append("momentum")
    # 3. shear-wave viscosity nu = cs2 (tau - 1/2)
    N, tau = 16, 0.8
    y = torch.arange(N, dtype=torch.float64).reshape(1, N, 1)
    mode = torch.sin(2 * math.pi * y / N)
    u = torch.zeros((3, 1, N, 1), dtype=torch.float64)
    u[0] = 1e-3 * mode
    Ms = synth.moments_from_velocity(torch.zeros((1, N, 1), dtype=torch.float64), u, tau)
    ts, amps = [], []
    lbm.run(lat, Ms, 40, tau, callback=lambda t, MM: (ts.append(t), amps.append(float((MM[1] * mode).sum()))))
    nu_fit = -dg.fit_decay_rate(ts, [abs(v) + 1e-300 for v in amps]) / (2 * math.pi / N) ** 2
    if not abs(nu_fit - CS2 * (tau - 0.5)) < 1e-2 * CS2 * (tau - 0.5):
        failed.append("viscosity")
    # 4. mass conservation with walls
    Mw = lbm.run(lat, M, 3, 0.75, force=F, solid=solid)
    if not abs(float(Mw[0][~solid].sum() - M[0][~solid].sum())) < 1e-15:
        failed.append("walls-mass")
    # 5. steady Poiseuille (short: H = 6, tau = 1.5 converges within ~300 steps)
    Hc, tc, g = 6, 1.5, 1e-5
    Mc, sc = synth.channel((1, Hc + 2, 1), 0.0, seed=0)
    Mc = lbm.run(lat, Mc, 300, tc, force=(g, 0.0, 0.0), solid=sc)
    eta = torch.arange(Hc + 2, dtype=torch.float64) - 0.5
    want = dg.poiseuille_steady(g, CS2 * (tc - 0.5), Hc, eta)[1:-1]
    if not float((Mc[1, 0, 1:-1, 0] - want).abs().max() / want.max()) < 5e-2:
        failed.append("poiseuille")
    return failed


def test_unmutated_oracle_passes_the_battery():
    assert pins_fail() == []


def _guo_wrong_sign(lat, u, F, rho):
    cu = torch.einsum("qa,a...->q...", lat.c, u)
    cF = torch.einsum("qa,a...->q...", lat.c, F)
    uF = (u * F).sum(0)
    return lbm._wq(lat, uF) * ((cF + uF.unsqueeze(0)) / CS2 + cu * cF / (CS2 * CS2)) / rho.unsqueeze(0)


def _collide_full_source(lat, f, F, rho, omega):
    p, u, A = lbm.macroscopic(lat, f, F, rho)
    uu = torch.einsum("a...,b...->ab...", u, u)
    feq = lbm.hermite_reconstruct(lat, p, u, uu)
    S = lbm.guo_source(lat, u, F, rho)
    _, _, a2neq = lbm.hermite_project(lat, f - feq + 0.5 * S)
    fneq = lbm.hermite_reconstruct(lat, torch.zeros_like(p), torch.zeros_like(u), a2neq)
    return feq + (1.0 - omega).unsqueeze(0) * fneq + S  # dropped the 1/2


def _collide_omega_not_one_minus(lat, f, F, rho, omega):
    p, u, A = lbm.macroscopic(lat, f, F, rho)
    uu = torch.einsum("a...,b...->ab...", u, u)
    feq = lbm.hermite_reconstruct(lat, p, u, uu)
    S = lbm.guo_source(lat, u, F, rho)
    _, _, a2neq = lbm.hermite_project(lat, f - feq + 0.5 * S)
    fneq = lbm.hermite_reconstruct(lat, torch.zeros_like(p), torch.zeros_like(u), a2neq)
    return feq + omega.unsqueeze(0) * fneq + 0.5 * S


def _collide_unregularized_total_a2(lat, f, F, rho, omega):
    p, u, A = lbm.macroscopic(lat, f, F, rho)
    uu = torch.einsum("a...,b...->ab...", u, u)
    feq = lbm.hermite_reconstruct(lat, p, u, uu)
    S = lbm.guo_source(lat, u, F, rho)
    fneq = lbm.hermite_reconstruct(lat, torch.zeros_like(p), torch.zeros_like(u), A)  # A, not A - uu
    return feq + (1.0 - omega).unsqueeze(0) * fneq + 0.5 * S


def _macroscopic_no_shift(lat, f, F, rho):
    a0, a1, a2 = lbm.hermite_project(lat, f)
    u = a1  # missing + F/(2 rho)
    uF = torch.einsum("a...,b...->ab...", u, F)
    return a0, u, a2 + (uF + uF.transpose(0, 1)) / (2.0 * rho)


def _macroscopic_no_tensor_shift(lat, f, F, rho):
    a0, a1, a2 = lbm.hermite_project(lat, f)
    return a0, a1 + F / (2.0 * rho), a2


def _stream_bounce_same_direction(lat, fpost, solid=None):
    out = torch.empty_like(fpost)
    for i in range(lat.Q):
        pulled = lbm.shift_from(fpost[i], lat.ci[i])
        if solid is not None:
            pulled = torch.where(lbm.shift_from(solid, lat.ci[i]), fpost[i], pulled)
        out[i] = pulled
    return out


def _shift_axes_transposed(x, c):
    return torch.roll(x, shifts=(int(c[0]), int(c[1]), int(c[2])), dims=(-3, -2, -1))


def _reconstruct_wrong_factor(lat, a0, a1, a2):
    t1 = torch.einsum("qa,a...->q...", lat.c, a1) / CS2
    t2 = torch.einsum("qab,ab...->q...", lat.H2, a2) / (CS2 * CS2)  # should be 2 cs2^2
    return lbm._wq(lat, a0) * (a0.unsqueeze(0) + t1 + t2)


def _populations_wrong_shift_sign(lat, M, F, rho):
    p, u, A = lbm.unpack(M)
    F = lbm.as_field(F, p.shape)
    rho = lbm.as_scalar_field(rho, p.shape)
    uF = torch.einsum("a...,b...->ab...", u, F)
    return lbm.hermite_reconstruct(lat, p, u + F / (2.0 * rho), A - (uF + uF.transpose(0, 1)) / (2.0 * rho))


MUTANTS = {
    "guo_source": _guo_wrong_sign,
    "collide_half_source": ("collide", _collide_full_source),
    "collide_omega": ("collide", _collide_omega_not_one_minus),
    "collide_regularization": ("collide", _collide_unregularized_total_a2),
    "macroscopic_velocity_shift": ("macroscopic", _macroscopic_no_shift),
    "macroscopic_tensor_shift": ("macroscopic", _macroscopic_no_tensor_shift),
    "stream_bounce_back": ("stream", _stream_bounce_same_direction),
    "shift_axes": ("shift_from", _shift_axes_transposed),
    "hermite_factor": ("hermite_reconstruct", _reconstruct_wrong_factor),
    "initial_shift_sign": ("populations_from_moments", _populations_wrong_shift_sign),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    target = MUTANTS[name]
    attr, fn = (name, target) if callable(target) else target
    monkeypatch.setattr(lbm, attr, fn)
    assert pins_fail() != [], f"mutant {name} passed every pin"


def test_planted_mistake_in_laplacian_factor_is_caught(monkeypatch):
    """Laplacian with factor 1/cs2 instead of 2/cs2: the flat-interface equilibrium moves away."""
    def lap_half(psi):
        acc = torch.zeros_like(psi)
        for i in range(oracle.D3Q27.Q):
            acc += oracle.D3Q27.w[i] * (phase.shift_to(psi, oracle.D3Q27.ci[i]) - psi)
        return acc / CS2
    monkeypatch.setattr(phase, "laplacian", lap_half)
    n, W = 32, 4.0
    x = torch.arange(n, dtype=torch.float64).reshape(1, 1, n)
    k = 2 * math.pi / n
    psi = torch.sin(k * x).expand(1, 1, n)
    assert (phase.laplacian(psi) + 4 * math.sin(k / 2) ** 2 * psi).abs().max() > 1e-4


def _pressure_force_dropped(phi, p, rho_l, rho_h):
    return torch.zeros((3,) + tuple(phi.shape), dtype=torch.float64)


def _pressure_force_sign(phi, p, rho_l, rho_h):
    return (CS2 * p).unsqueeze(0) * ((rho_h - rho_l) * phase.gradient(phi))


def _pressure_force_no_cs2(phi, p, rho_l, rho_h):
    return -p.unsqueeze(0) * ((rho_h - rho_l) * phase.gradient(phi))


@pytest.mark.parametrize("mutant", [_pressure_force_dropped, _pressure_force_sign, _pressure_force_no_cs2],
                         ids=["dropped", "sign", "no_cs2"])
def test_planted_mistake_in_pressure_force_is_caught(mutant, monkeypatch):
    """F_p = -p* cs2 grad rho (Sec. 2): dropping it, flipping its sign or losing the cs2 breaks the
    rest state of a density interface at uniform physical pressure."""
    from test_oracle_pressure_force import pressure_pin_holds

    assert pressure_pin_holds()
    monkeypatch.setattr(phase, "pressure_force", mutant)
    assert not pressure_pin_holds()
