"""Pins of the oracle's gradients (oracle.adjoint) by central finite differences of the oracle's
own forward map and by the dot-product identity <J v, w> = <v, J^T w> for one step."""
import pytest
import torch

import oracle
import synth
from oracle import adjoint, lbm

LATS = [oracle.D3Q19, oracle.D3Q27]
ids = lambda l: l.name  # noqa: E731


def small_channel(seed=0):
    shape = (4, 7, 5)
    M0 = synth.random_moments(shape, seed=seed, p_scale=1e-3, u_scale=0.02, neq_scale=1e-4)
    solid = synth.channel_walls(shape)
    F = synth.random_field(shape, 1e-4, seed=seed + 1, mask=solid)
    u_tgt = synth.random_field(shape, 1e-3, seed=seed + 2)
    return M0, F, solid, u_tgt


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_step_vjp_dot_product(lat):
    M0, F, solid, _ = small_channel(5)
    g = torch.Generator().manual_seed(9)
    v = torch.randn(M0.shape, dtype=torch.float64, generator=g) * 1e-4
    vF = torch.randn(F.shape, dtype=torch.float64, generator=g) * 1e-5
    w = torch.randn(M0.shape, dtype=torch.float64, generator=g)
    lam, gF = adjoint.step_vjp(lat, M0, 0.7, F, w, solid)
    eps = 1e-3
    plus = lbm.step_moments(lat, M0 + eps * v, 0.7, F + eps * vF, F + eps * vF, solid)
    minus = lbm.step_moments(lat, M0 - eps * v, 0.7, F - eps * vF, F - eps * vF, solid)
    jv = (plus - minus) / (2 * eps)
    lhs = float((jv * w).sum())
    rhs = float((v * lam).sum() + (vF * gF).sum())
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_rollout_gradient_matches_central_differences(lat):
    M0, F, solid, u_tgt = small_channel(7)
    steps, tau = 6, 0.7
    L, gM, gF = adjoint.rollout_gradient(lat, M0, F, steps, tau, u_tgt, solid)
    assert float(L) > 0
    picks = [("F", (0, 1, 2, 3)), ("F", (1, 2, 5, 1)), ("F", (2, 0, 3, 4)),
             ("M", (1, 2, 3, 2)), ("M", (0, 1, 1, 1)), ("M", (7, 3, 4, 0)), ("M", (5, 0, 2, 2))]
    for which, idx in picks:
        base = F if which == "F" else M0
        eps = 1e-6 * max(float(base.abs().max()), 1e-3)
        bp, bm = base.clone(), base.clone()
        bp[idx] += eps
        bm[idx] -= eps
        if which == "F":
            lp = adjoint.rollout_loss(lat, M0, bp, steps, tau, u_tgt, solid)
            lm = adjoint.rollout_loss(lat, M0, bm, steps, tau, u_tgt, solid)
            got = gF[idx]
        else:
            lp = adjoint.rollout_loss(lat, bp, F, steps, tau, u_tgt, solid)
            lm = adjoint.rollout_loss(lat, bm, F, steps, tau, u_tgt, solid)
            got = gM[idx]
        fd = float(lp - lm) / (2 * eps)
        scale = max(abs(fd), 1e-6 * float(gF.abs().max() if which == "F" else gM.abs().max()))
        assert abs(float(got) - fd) < 1e-5 * scale, (which, idx, float(got), fd)
