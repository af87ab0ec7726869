"""Pins of the D3Q27h oracle: the D3Q27 velocity set with its complete Hermite basis and the
recursive closure of the higher-order non-equilibrium coefficients (Sec. 2).

Each pin is fixed by something other than the oracle's own formula: the orthogonality of the
basis under the quadrature, the closed product form of the full equilibrium, the reduction to the
second-order scheme where every higher-order coefficient vanishes, the conservation of the
moments the step keeps, the Malaspinas recursion (an independent formula for the closure) and the
physics the higher-order terms exist for: a shear wave advected at speed U decays with the
viscosity nu for D3Q27h, while the second-order D3Q27 scheme decays with nu (1 - 3 U^2) because
its equilibrium lacks the third moment u_x u_x u_y.
"""
import math

import torch

import oracle
from oracle import lbm
from oracle.lattice import CS2, MULTI, axes_of


def _random_state(shape, seed, scale=1e-2):
    g = torch.Generator().manual_seed(seed)
    M = scale * torch.randn((10,) + shape, generator=g, dtype=torch.float64)
    F = 1e-3 * torch.randn((3,) + shape, generator=g, dtype=torch.float64)
    return M, F


def test_full_basis_is_orthogonal_under_the_d3q27_weights():
    lat = oracle.D3Q27H
    gram = torch.einsum("mi,i,ni->mn", lat.HM, lat.w, lat.HM)
    want = torch.diag(torch.tensor([math.prod(math.factorial(k) * CS2 ** k for k in m) for m in MULTI],
                                   dtype=torch.float64))
    assert torch.allclose(gram, want, atol=1e-15, rtol=0)
    # the basis spans the 27 populations: reconstruct(project(f)) = f
    f = torch.randn(27, dtype=torch.float64)
    back = lat.w * (lat.HM.T @ ((lat.HM @ f) / lat.HM_norm))
    assert torch.allclose(back, f, atol=1e-13)


def test_full_equilibrium_has_the_closed_product_form():
    """N = 0 and F = 0: f_i = w_i [p* - 1 + prod_a (1 + c_a u_a / cs2 + (c_a^2 - cs2) u_a^2 / (2 cs2^2))]."""
    lat = oracle.D3Q27H
    shape = (2, 3, 4)
    M, _ = _random_state(shape, 1, scale=5e-2)
    u = M[1:4]
    M[4], M[5], M[6] = u[0] * u[0], u[1] * u[1], u[2] * u[2]
    M[7], M[8], M[9] = u[0] * u[1], u[0] * u[2], u[1] * u[2]
    zero = torch.zeros((3,) + shape, dtype=torch.float64)
    rho = torch.ones(shape, dtype=torch.float64)
    om = torch.full(shape, 1.7, dtype=torch.float64)
    f = lbm.populations_from_moments(lat, M, zero, rho)
    got = lbm.collide(lat, f, zero, rho, om)
    prod = torch.ones((27,) + shape, dtype=torch.float64)
    for a in range(3):
        c = lat.c[:, a].reshape((27, 1, 1, 1))
        ua = u[a].unsqueeze(0)
        prod = prod * (1 + c * ua / CS2 + (c * c - CS2) * ua * ua / (2 * CS2 * CS2))
    want = lat.w.reshape((27, 1, 1, 1)) * (M[0].unsqueeze(0) - 1 + prod)
    assert torch.allclose(got, want, atol=1e-15, rtol=1e-13)


def test_reduces_to_the_second_order_scheme_without_velocity():
    """Every coefficient beyond second order carries a factor u, so at u = 0 and F = 0 the D3Q27h
    collision equals the second-order D3Q27 one."""
    shape = (3, 2, 5)
    M, _ = _random_state(shape, 2)
    M[1:4] = 0.0
    zero = torch.zeros((3,) + shape, dtype=torch.float64)
    rho = torch.ones(shape, dtype=torch.float64)
    om = torch.full(shape, 1.2, dtype=torch.float64)
    f = lbm.populations_from_moments(oracle.D3Q27, M, zero, rho)
    a = lbm.collide(oracle.D3Q27, f, zero, rho, om)
    b = lbm.collide(oracle.D3Q27H, f, zero, rho, om)
    assert torch.allclose(a, b, atol=1e-17, rtol=0)


def test_higher_orders_leave_the_kept_moments_unchanged():
    """The added terms are orthogonal to H0, H1, H2: mass, momentum and the second moment of the
    post-collision populations are those of the second-order scheme; the higher moments differ."""
    shape = (2, 2, 3)
    M, F = _random_state(shape, 3, scale=4e-2)
    rho = torch.ones(shape, dtype=torch.float64)
    om = torch.full(shape, 1.6, dtype=torch.float64)
    f = lbm.populations_from_moments(oracle.D3Q27, M, F, rho)
    a = lbm.collide(oracle.D3Q27, f, F, rho, om)
    b = lbm.collide(oracle.D3Q27H, f, F, rho, om)
    for x, y in zip(lbm.hermite_project(oracle.D3Q27, a), lbm.hermite_project(oracle.D3Q27, b)):
        assert torch.allclose(x, y, atol=1e-16, rtol=1e-13)
    assert float((a - b).abs().max()) > 1e-6


def test_closure_matches_the_malaspinas_recursion():
    """The pair sum of the oracle against the recursion
    a(a1..an) = u_an a(a1..a(n-1)) + sum_{i<n} (prod_{j<n, j != i} u_aj) N_(ai an), started at a2 = N."""
    g = torch.Generator().manual_seed(4)
    u = torch.randn(3, 1, generator=g, dtype=torch.float64)
    N = torch.randn(3, 3, 1, generator=g, dtype=torch.float64)
    N = 0.5 * (N + N.transpose(0, 1))
    p = torch.zeros(1, dtype=torch.float64)
    zero = torch.zeros(3, 1, dtype=torch.float64)
    coefs = lbm.full_coefficients(oracle.D3Q27H, p, u, N, zero, torch.ones(1, dtype=torch.float64),
                                  torch.zeros(1, dtype=torch.float64))  # omega = 0: P = a_eq + a_neq

    def rec(al):
        if len(al) == 2:
            return N[al[0], al[1]]
        n = len(al)
        out = u[al[-1]] * rec(al[:-1])
        for i in range(n - 1):
            pr = torch.ones(1, dtype=torch.float64)
            for j in range(n - 1):
                if j != i:
                    pr = pr * u[al[j]]
            out = out + pr * N[al[i], al[-1]]
        return out

    for m, c in zip(MULTI, coefs):
        al = axes_of(m)
        if len(al) < 3:
            continue
        eq = torch.ones(1, dtype=torch.float64)
        for a in al:
            eq = eq * u[a]
        assert torch.allclose(c - eq, rec(al), atol=1e-14, rtol=1e-12), m


def _shear_wave_viscosity(lat, U, tau=0.6, nx=32, steps=300, amp=1e-3):
    """Decay rate / k^2 of a shear wave u_y = amp sin(k x) advected by u_x = U (periodic)."""
    shape = (2, 2, nx)
    x = torch.arange(nx, dtype=torch.float64)
    k = 2 * math.pi / nx
    M = torch.zeros((10,) + shape, dtype=torch.float64)
    M[1] = U
    M[2] = amp * torch.sin(k * x)
    M[4] = M[1] * M[1]
    M[5] = M[2] * M[2]
    M[7] = M[1] * M[2] - CS2 * tau * amp * k * torch.cos(k * x)  # Chapman-Enskog shear stress
    amps = []
    lbm.run(lat, M, steps, tau, callback=lambda t, Mt: amps.append(abs(complex(torch.fft.fft(Mt[2, 0, 0])[1]))))
    return math.log(amps[49] / amps[-1]) / (len(amps) - 50) / k ** 2


def test_shear_viscosity_is_galilean_invariant_with_the_full_basis():
    """At U = 0.15 the second-order D3Q27 scheme decays with nu (1 - 3 U^2) (its equilibrium lacks
    the supported third moment u_x u_x u_y); D3Q27h keeps the viscosity of the wave at rest."""
    U = 0.15
    r27 = _shear_wave_viscosity(oracle.D3Q27, U) / _shear_wave_viscosity(oracle.D3Q27, 0.0)
    assert abs(r27 - (1 - 3 * U * U)) < 3e-3, r27
    r27h = _shear_wave_viscosity(oracle.D3Q27H, U) / _shear_wave_viscosity(oracle.D3Q27H, 0.0)
    assert abs(r27h - 1) < 1e-3, r27h


def test_forcing_is_expanded_to_the_same_orders():
    """With N = 0 the coefficients are u^m + S_m / 2 = (u + F / (2 rho))^m - O(F^2): the
    post-collision populations equal the product-form equilibrium at the half-force-shifted
    velocity up to O(F^2). A source truncated at second order leaves an O(F u^2) difference."""
    lat = oracle.D3Q27H
    shape = (2, 2, 2)
    g = torch.Generator().manual_seed(5)
    u = 0.1 * torch.randn((3,) + shape, generator=g, dtype=torch.float64)
    F = 1e-4 * torch.randn((3,) + shape, generator=g, dtype=torch.float64)
    rho = torch.ones(shape, dtype=torch.float64)
    p = 1e-3 * torch.randn(shape, generator=g, dtype=torch.float64)
    zeroN = torch.zeros((3, 3) + shape, dtype=torch.float64)
    got = lbm.full_reconstruct(lat, lbm.full_coefficients(lat, p, u, zeroN, F, rho, torch.ones(shape, dtype=torch.float64)))
    us = u + F / 2
    prod = torch.ones((27,) + shape, dtype=torch.float64)
    for a in range(3):
        c = lat.c[:, a].reshape((27, 1, 1, 1))
        prod = prod * (1 + c * us[a] / CS2 + (c * c - CS2) * us[a] * us[a] / (2 * CS2 * CS2))
    want = lat.w.reshape((27, 1, 1, 1)) * (p - 1 + prod)
    assert float((got - want).abs().max()) < 1e-8


# -- planted mistakes: each mutant of the D3Q27h oracle must fail at least one pin above -------
def _battery(monkeypatch_ctx=None):
    failed = []
    for name, fn in (("product", test_full_equilibrium_has_the_closed_product_form),
                     ("recursion", test_closure_matches_the_malaspinas_recursion),
                     ("forcing", test_forcing_is_expanded_to_the_same_orders),
                     ("moments", test_higher_orders_leave_the_kept_moments_unchanged),
                     ("reduction", test_reduces_to_the_second_order_scheme_without_velocity)):
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def _mutant_coefficients(kind):
    good = lbm.full_coefficients

    def coefs(lat, p, u, a2neq, F, rho, omega):
        out = []
        for m, c in zip(MULTI, good(lat, p, u, a2neq, F, rho, omega)):
            al = axes_of(m)
            n = len(al)
            if n >= 3 and kind == "closure-double-count":
                # recursion over single positions without removing repeated pairs: 2x at n >= 4
                extra = torch.zeros_like(p)
                for i in range(n):
                    for j in range(i + 1, n):
                        rest = [u[al[k]] for k in range(n) if k not in (i, j)]
                        t = a2neq[al[i], al[j]]
                        for v in rest:
                            t = t * v
                        extra = extra + t
                c = c + ((1.0 - omega) * extra if n >= 4 else 0.0)
            if n >= 3 and kind == "source-truncated":
                src = torch.zeros_like(p)
                for i in range(n):
                    t = F[al[i]]
                    for k in range(n):
                        if k != i:
                            t = t * u[al[k]]
                    src = src + t
                c = c - 0.5 * src / rho
            if n == 3 and kind == "eq-third-sign":
                c = c - 2 * u[al[0]] * u[al[1]] * u[al[2]]
            out.append(c)
        return out

    return coefs


def _mutant_norm_reconstruct(lat, coefs):
    """Hermite normalisation n! cs2^n instead of prod m_a! cs2^m_a."""
    P = torch.stack(coefs, dim=0)
    norm = torch.tensor([math.factorial(sum(m)) * CS2 ** sum(m) for m in MULTI], dtype=torch.float64)
    g = torch.einsum("mq,m...->q...", lat.HM / norm.unsqueeze(1), P)
    return lbm._wq(lat, coefs[0]) * g


def test_unmutated_d3q27h_oracle_passes_its_battery():
    assert _battery() == []


def test_planted_d3q27h_mistakes_are_caught(monkeypatch):
    for kind in ("closure-double-count", "source-truncated", "eq-third-sign"):
        with monkeypatch.context() as mp:
            mp.setattr(lbm, "full_coefficients", _mutant_coefficients(kind))
            assert _battery() != [], kind
    with monkeypatch.context() as mp:
        mp.setattr(lbm, "full_reconstruct", _mutant_norm_reconstruct)
        assert _battery() != [], "norm"
