"""Pins of the oracle's velocity sets, Hermite basis and Guo source against identities that the
quadrature and the paper's Hermite formulation must satisfy (Sec. 2)."""
import itertools

import pytest
import torch

import oracle
from oracle import lbm
from oracle.lattice import CS2

LATS = [oracle.D3Q19, oracle.D3Q27]
EYE = torch.eye(3, dtype=torch.float64)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_counts_and_opposites(lat):
    assert lat.Q == {"D3Q19": 19, "D3Q27": 27}[lat.name]
    assert torch.equal(lat.ci[lat.opp], -lat.ci)
    assert len({tuple(v.tolist()) for v in lat.ci}) == lat.Q


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_isotropy_up_to_fourth_order(lat):
    c, w = lat.c, lat.w
    assert torch.isclose(w.sum(), torch.tensor(1.0, dtype=torch.float64), atol=1e-15)
    assert torch.allclose(torch.einsum("q,qa->a", w, c), torch.zeros(3, dtype=torch.float64), atol=1e-15)
    assert torch.allclose(torch.einsum("q,qa,qb->ab", w, c, c), CS2 * EYE, atol=1e-15)
    third = torch.einsum("q,qa,qb,qc->abc", w, c, c, c)
    assert third.abs().max() < 1e-15
    fourth = torch.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    iso = (torch.einsum("ab,cd->abcd", EYE, EYE) + torch.einsum("ac,bd->abcd", EYE, EYE)
           + torch.einsum("ad,bc->abcd", EYE, EYE)) * CS2 * CS2
    assert (fourth - iso).abs().max() < 1e-15


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_hermite_orthogonality(lat):
    """sum_i w_i H^(m)_i H^(n)_i = 0 for m != n and cs2^n n! (symmetrised identity) for m = n <= 2."""
    w, c, H2 = lat.w, lat.c, lat.H2
    assert torch.allclose(torch.einsum("q,qa->a", w, c), torch.zeros(3, dtype=torch.float64), atol=1e-15)
    assert torch.einsum("q,qab->ab", w, H2).abs().max() < 1e-15
    assert torch.einsum("q,qa,qbc->abc", w, c, H2).abs().max() < 1e-15
    g = torch.einsum("q,qab,qcd->abcd", w, H2, H2)
    want = CS2 * CS2 * (torch.einsum("ac,bd->abcd", EYE, EYE) + torch.einsum("ad,bc->abcd", EYE, EYE))
    assert (g - want).abs().max() < 1e-15


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_reconstruct_then_project_is_identity(lat):
    torch.manual_seed(0)
    shape = (3, 2, 2)
    a0 = torch.randn(shape, dtype=torch.float64)
    a1 = torch.randn((3,) + shape, dtype=torch.float64)
    B = torch.randn((3, 3) + shape, dtype=torch.float64)
    a2 = B + B.transpose(0, 1)
    b0, b1, b2 = lbm.hermite_project(lat, lbm.hermite_reconstruct(lat, a0, a1, a2))
    assert torch.allclose(b0, a0, atol=1e-14)
    assert torch.allclose(b1, a1, atol=1e-14)
    assert torch.allclose(b2, a2, atol=1e-14)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_guo_source_moments(lat):
    """Moments of Eq. (guoforce): sum S = 0, sum c S = F/rho, sum H2 S = (u F + F u)/rho."""
    torch.manual_seed(1)
    shape = (4,)
    u = 0.1 * torch.randn((3,) + shape, dtype=torch.float64)
    F = 1e-2 * torch.randn((3,) + shape, dtype=torch.float64)
    rho = 1.0 + 0.3 * torch.rand(shape, dtype=torch.float64)
    S = lbm.guo_source(lat, u, F, rho)
    s0, s1, s2 = lbm.hermite_project(lat, S)
    uF = torch.einsum("a...,b...->ab...", u, F)
    assert s0.abs().max() < 1e-16
    assert torch.allclose(s1, F / rho, atol=1e-16)
    assert torch.allclose(s2, (uF + uF.transpose(0, 1)) / rho, atol=1e-16)


def test_textbook_weights():
    """Weights of the textbook quadratures, grouped by |c|^2."""
    for lat, want in ((oracle.D3Q19, {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}),
                      (oracle.D3Q27, {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216})):
        for i in range(lat.Q):
            n2 = int((lat.ci[i] ** 2).sum())
            assert abs(float(lat.w[i]) - want[n2]) < 1e-16


def test_d3q19_is_the_d3q27_subset_without_corners():
    v19 = {tuple(v.tolist()) for v in oracle.D3Q19.ci}
    v27 = {tuple(v.tolist()) for v in oracle.D3Q27.ci}
    corners = {v for v in itertools.product((-1, 1), repeat=3)}
    assert v27 - v19 == corners
