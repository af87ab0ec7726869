"""Pins of the oracle's step map: fixed points, conservation, lattice symmetry, the brute-force
agreement between the population form and the literal moment form of Eq. (pullLLB), and the
site-sampled variant used for full-size checks."""
import pytest
import torch

import oracle
import synth
from oracle import lbm, moment_form

LATS = [oracle.D3Q19, oracle.D3Q27]
ids = lambda l: l.name  # noqa: E731


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp(min=1e-300))


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_rest_state_is_a_fixed_point(lat):
    M = torch.zeros((10, 3, 4, 5), dtype=torch.float64)
    assert lbm.run(lat, M, 3, 0.7).abs().max() == 0.0
    M[0] = 2.5e-3  # uniform pressure, fluid at rest
    out = lbm.run(lat, M, 3, 0.7)
    assert (out - M).abs().max() < 1e-18


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_uniform_flow_stays_uniform(lat):
    u0 = torch.tensor([0.03, -0.02, 0.01], dtype=torch.float64)
    shape = (3, 4, 5)
    p = torch.full(shape, 1e-3, dtype=torch.float64)
    u = u0.reshape(3, 1, 1, 1).expand((3,) + shape)
    A = torch.einsum("a...,b...->ab...", u, u)
    M = lbm.pack(p, u, A)
    out = lbm.run(lat, M, 4, 0.6)
    assert rel(out, M) < 1e-13


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_mass_and_momentum_conserved_periodic(lat):
    M0 = synth.random_moments((5, 6, 7), seed=11)
    M = lbm.run(lat, M0, 6, 0.62)
    assert abs(float(M[0].sum() - M0[0].sum())) < 1e-15
    assert (M[1:4].sum((1, 2, 3)) - M0[1:4].sum((1, 2, 3))).abs().max() < 1e-15
    assert rel(M, M0) > 1e-3  # the state did evolve


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_momentum_grows_by_total_force(lat):
    """sum u(t+1) = sum u(t) + N F / rho on a periodic box with uniform force."""
    M0 = synth.random_moments((4, 5, 6), seed=12)
    F = torch.tensor([1e-4, -2e-4, 3e-5], dtype=torch.float64)
    n = 4 * 5 * 6
    M = lbm.run(lat, M0, 5, 0.7, force=F)
    grow = M[1:4].sum((1, 2, 3)) - M0[1:4].sum((1, 2, 3))
    assert (grow - 5 * n * F).abs().max() < 1e-15
    assert abs(float(M[0].sum() - M0[0].sum())) < 1e-15


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_bounce_back_conserves_mass(lat):
    shape = (6, 7, 5)
    M0 = synth.random_moments(shape, seed=13)
    solid = synth.random_mask(shape, 0.25, seed=14)
    F = synth.random_field(shape, 1e-4, seed=15, mask=solid)
    M = lbm.run(lat, M0, 5, 0.75, force=F, solid=solid)
    fluid = ~solid
    assert abs(float(M[0][fluid].sum() - M0[0][fluid].sum())) < 1e-15
    assert torch.equal(M[:, solid], M0[:, solid])


def _swap_xy(M, F=None, solid=None):
    """Apply the lattice symmetry x <-> y to a state (field axes and tensor components)."""
    p, u, A = lbm.unpack(M)
    perm = [1, 0, 2]
    u2 = u[perm].transpose(-1, -2)
    A2 = A[perm][:, perm].transpose(-1, -2)
    out = [lbm.pack(p.transpose(-1, -2), u2, A2)]
    if F is not None:
        out.append(F[perm].transpose(-1, -2))
    if solid is not None:
        out.append(solid.transpose(-1, -2))
    return out


def _mirror_x(M, F=None, solid=None):
    """x -> -x (site index i -> (-i) mod nx): u_x, A_xy, A_xz change sign."""
    def flip(t):
        return torch.roll(torch.flip(t, dims=(-1,)), shifts=1, dims=-1)
    p, u, A = lbm.unpack(M)
    s = torch.tensor([-1.0, 1.0, 1.0], dtype=torch.float64)
    u2 = flip(u * s.reshape(3, 1, 1, 1))
    A2 = flip(A * torch.einsum("a,b->ab", s, s).reshape(3, 3, 1, 1, 1))
    out = [lbm.pack(flip(p), u2, A2)]
    if F is not None:
        out.append(flip(F * s.reshape(3, 1, 1, 1)))
    if solid is not None:
        out.append(flip(solid))
    return out


@pytest.mark.parametrize("lat", LATS, ids=ids)
@pytest.mark.parametrize("sym", [_swap_xy, _mirror_x], ids=["swap_xy", "mirror_x"])
def test_lattice_symmetry_equivariance(lat, sym):
    shape = (4, 6, 6)
    M0 = synth.random_moments(shape, seed=21)
    solid = synth.random_mask(shape, 0.15, seed=22)
    F = synth.random_field(shape, 1e-3, seed=23, mask=solid)
    out = lbm.run(lat, M0, 3, 0.66, force=F, solid=solid)
    Ms, Fs, ss = sym(M0, F, solid)
    out_s = lbm.run(lat, Ms, 3, 0.66, force=Fs, solid=ss)
    assert rel(out_s, sym(out)[0]) < 1e-13


@pytest.mark.parametrize("lat", LATS, ids=ids)
@pytest.mark.parametrize("walls", [False, True])
def test_population_form_equals_literal_moment_form(lat, walls):
    """Brute force on a 4^3 box: Eq. (pullLLB) + Eq. (corr) evaluated literally, site by site,
    gives the same moments as the population-form step, for several steps."""
    shape = (4, 4, 4)
    M = synth.random_moments(shape, seed=31)
    F = synth.random_field(shape, 1e-3, seed=32)
    solid = synth.random_mask(shape, 0.2, seed=33) if walls else None
    Mp = M.clone()
    Ml = M.tolist()
    for _ in range(3):
        Mp = lbm.step_moments(lat, Mp, 0.7, F, F, solid)
        Ml = moment_form.step(lat, Ml, 0.7, F.tolist(), F.tolist(),
                              None if solid is None else solid.tolist())
    assert rel(torch.tensor(Ml, dtype=torch.float64), Mp) < 1e-13


@pytest.mark.parametrize("lat", LATS, ids=ids)
def test_step_at_sites_matches_full_step(lat):
    shape = (5, 7, 9)
    M = synth.random_moments(shape, seed=41)
    solid = synth.random_mask(shape, 0.2, seed=42)
    F = synth.random_field(shape, 1e-3, seed=43, mask=solid)
    full = lbm.step_moments(lat, M, 0.8, F, F, solid)
    sites = torch.tensor([[0, 0, 0], [4, 6, 8], [2, 3, 4], [1, 0, 8], [3, 6, 0]])
    got = lbm.step_at_sites(lat, M, sites, 0.8, F, solid)
    want = full[:, sites[:, 0], sites[:, 1], sites[:, 2]]
    assert rel(got, want) < 1e-14
    got_u = lbm.step_at_sites(lat, M, sites, 0.8, torch.tensor([1e-4, 0.0, -1e-4]), None)
    full_u = lbm.step_moments(lat, M, 0.8, torch.tensor([1e-4, 0.0, -1e-4]))
    assert rel(got_u, full_u[:, sites[:, 0], sites[:, 1], sites[:, 2]]) < 1e-14
