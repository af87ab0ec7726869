"""Population-form FP64 reference of the regularized pull lattice Boltzmann step.

TEST INFRASTRUCTURE. This module is the oracle: it is imported only by the tests, by the
smoke check and by the CPU-baseline legs of the benchmark script, never by the library.

What it computes (Sec. 2 of the paper, velocity-pressure formulation):

* populations are stored explicitly, one FP64 field per direction;
* Eq. (hermite_teq): Hermite coefficients by projection, a0 = sum f, a1 = sum c f,
  a2 = sum (c c - cs2 delta) f;
* Eq. (corr): the stored velocity and second moment carry the half-force shift,
  u = a1 + F/(2 rho), A = a2 + (F u + u F)/(2 rho);
* velocity form of the equilibrium coefficients: a_eq = (p*, u, u u);
* f_neq = f - f_eq + S/2 (text under Eq. pullLB) projected on the Hermite basis and truncated
  at second order (a0_neq = a1_neq = 0), which is the regularization;
* Eq. (guoforce): Guo source S_i;
* Eq. (pullLB): f_i(x, t+1) = f_eq_i + (1 - omega) f_neq_i + S_i/2, all taken at x - c_i;
* walls: halfway bounce-back (the paper only says "no-slip walls"): when x - c_i is solid,
  f_i(x, t+1) is the post-collision population of the opposite direction at x itself.

Field layout of a moment state M (the public layout): shape (10, nz, ny, nx), FP64,
components [p*, ux, uy, uz, Axx, Ayy, Azz, Axy, Axz, Ayz], with A the total second-order
Hermite coefficient a^(2).
"""
import torch

from .lattice import CS2

# (row, col) of the six stored components of the symmetric tensor A, in storage order
SYM = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def unpack(M):
    """Split a (10, ...) moment state into p* (...), u (3, ...), A (3, 3, ...)."""
    p = M[0]
    u = M[1:4]
    A = torch.empty((3, 3) + tuple(M.shape[1:]), dtype=M.dtype)
    for k, (a, b) in enumerate(SYM):
        A[a, b] = M[4 + k]
        A[b, a] = M[4 + k]
    return p, u, A


def pack(p, u, A):
    """Inverse of unpack (uses the upper triangle of A)."""
    comps = [p, u[0], u[1], u[2]] + [A[a, b] for (a, b) in SYM]
    return torch.stack(comps, dim=0)


def _wq(lat, like):
    """Weights reshaped to (Q, 1, 1, ...) for broadcasting against fields shaped like `like`."""
    return lat.w.reshape((lat.Q,) + (1,) * like.dim())


def as_field(v, shape):
    """Uniform 3-vector (3,) or field (3, *shape) -> field (3, *shape) (broadcast view)."""
    v = torch.as_tensor(v, dtype=torch.float64)
    if v.dim() == 1:
        return v.reshape((3,) + (1,) * len(shape)).expand((3,) + tuple(shape))
    return v


def as_scalar_field(v, shape):
    v = torch.as_tensor(v, dtype=torch.float64)
    if v.dim() == 0:
        return v.expand(tuple(shape))
    return v


def hermite_reconstruct(lat, a0, a1, a2):
    """Truncated Hermite expansion, Eq. (reqfeq)/(reqfneq) with n <= 2:
    f_i = w_i [ a0 + H1_i . a1 / cs2 + H2_i : a2 / (2 cs2^2) ]."""
    t1 = torch.einsum("qa,a...->q...", lat.c, a1) / CS2
    t2 = torch.einsum("qab,ab...->q...", lat.H2, a2) / (2.0 * CS2 * CS2)
    return _wq(lat, a0) * (a0.unsqueeze(0) + t1 + t2)


def hermite_project(lat, f):
    """Hermite coefficients by projection, Eq. (hermite_teq): sum_i H^(n)_i f_i for n = 0, 1, 2."""
    a0 = f.sum(0)
    a1 = torch.einsum("qa,q...->a...", lat.c, f)
    a2 = torch.einsum("qab,q...->ab...", lat.H2, f)
    return a0, a1, a2


def guo_source(lat, u, F, rho):
    """Eq. (guoforce): S_i = w_i [ (c_i - u) . F / cs2 + (c_i . u)(c_i . F) / cs2^2 ] / rho."""
    cu = torch.einsum("qa,a...->q...", lat.c, u)
    cF = torch.einsum("qa,a...->q...", lat.c, F)
    uF = (u * F).sum(0)
    return _wq(lat, uF) * ((cF - uF.unsqueeze(0)) / CS2 + cu * cF / (CS2 * CS2)) / rho.unsqueeze(0)


def macroscopic(lat, f, F, rho):
    """Stored variables from populations: projection then the Eq. (corr) half-force shift.
    Returns p* (...), u (3, ...), A (3, 3, ...)."""
    a0, a1, a2 = hermite_project(lat, f)
    u = a1 + F / (2.0 * rho)
    uF = torch.einsum("a...,b...->ab...", u, F)
    A = a2 + (uF + uF.transpose(0, 1)) / (2.0 * rho)
    return a0, u, A


def populations_from_moments(lat, M, F, rho):
    """Populations whose Hermite moments, after the Eq. (corr) shift with force F, equal M.
    The shift is undone first, then the truncated expansion is evaluated."""
    p, u, A = unpack(M)
    shape = p.shape
    F = as_field(F, shape)
    rho = as_scalar_field(rho, shape)
    uF = torch.einsum("a...,b...->ab...", u, F)
    a1 = u - F / (2.0 * rho)
    a2 = A - (uF + uF.transpose(0, 1)) / (2.0 * rho)
    return hermite_reconstruct(lat, p, a1, a2)


def moments_from_populations(lat, f, F, rho):
    shape = f.shape[1:]
    p, u, A = macroscopic(lat, f, as_field(F, shape), as_scalar_field(rho, shape))
    return pack(p, u, A)


def _prod(fields, like):
    out = torch.ones_like(like)
    for v in fields:
        out = out * v
    return out


def full_coefficients(lat, p, u, a2neq, F, rho, omega):
    """Post-collision Hermite coefficients of D3Q27h for every multi-index m of the complete
    D3Q27 basis (Sec. 2, higher-order formulation with the recursive closure of Shan et al. and
    Malaspinas), in the velocity-pressure form of the paper. With alpha = axes_of(m), n = |alpha|:
      equilibrium      a_eq(m)  = p* (n = 0), u_alpha1 ... u_alphan (n >= 1)
      non-equilibrium  a_neq(m) = 0 (n < 2), N_alpha1alpha2 (n = 2), and for n >= 3 the closure
                       sum over index pairs {i, j} of N_alphai alphaj prod_{k not i, j} u_alphak
      Guo source       S(m)     = sum over positions i of F_alphai prod_{k != i} u_alphak / rho
    and P(m) = a_eq + (1 - omega) a_neq + S/2 (the bracket of Eq. pullLB). Truncated at n <= 2
    this is exactly the second-order scheme of `collide`. Returns a list in MULTI order."""
    from .lattice import MULTI, axes_of
    coefs = []
    for m in MULTI:
        al = axes_of(m)
        n = len(al)
        if n == 0:
            coefs.append(p)
            continue
        eq = _prod([u[a] for a in al], p)
        if n < 2:
            neq = torch.zeros_like(p)
        else:
            neq = torch.zeros_like(p)
            for i in range(n):
                for j in range(i + 1, n):
                    rest = [u[al[k]] for k in range(n) if k != i and k != j]
                    neq = neq + a2neq[al[i], al[j]] * _prod(rest, p)
        src = torch.zeros_like(p)
        for i in range(n):
            rest = [u[al[k]] for k in range(n) if k != i]
            src = src + F[al[i]] * _prod(rest, p)
        src = src / rho
        coefs.append(eq + (1.0 - omega) * neq + 0.5 * src)
    return coefs


def full_reconstruct(lat, coefs):
    """f_i = w_i sum_m H_m(c_i) P(m) / norm(m) over the complete D3Q27 basis."""
    P = torch.stack(coefs, dim=0)
    g = torch.einsum("mq,m...->q...", lat.HM / lat.HM_norm.unsqueeze(1), P)
    return _wq(lat, coefs[0]) * g


def collide(lat, f, F, rho, omega):
    """Right-hand side of Eq. (pullLB) at every site, before streaming:
    f_post = f_eq + (1 - omega) f_neq + S/2 with the regularized f_neq (second order), or the
    same bracket over the complete Hermite basis for D3Q27h (lat.high)."""
    if lat.high:
        p, u, A = macroscopic(lat, f, F, rho)
        uu = torch.einsum("a...,b...->ab...", u, u)
        S = guo_source(lat, u, F, rho)
        fneq_raw = f - hermite_reconstruct(lat, p, u, uu) + 0.5 * S
        _, _, a2neq = hermite_project(lat, fneq_raw)  # = A - u u
        return full_reconstruct(lat, full_coefficients(lat, p, u, a2neq, F, rho, omega))
    p, u, A = macroscopic(lat, f, F, rho)
    uu = torch.einsum("a...,b...->ab...", u, u)
    feq = hermite_reconstruct(lat, p, u, uu)  # a_eq = (p*, u, u u)
    S = guo_source(lat, u, F, rho)
    fneq_raw = f - feq + 0.5 * S  # definition under Eq. (pullLB)
    _, _, a2neq = hermite_project(lat, fneq_raw)
    zero = torch.zeros_like(p)
    fneq = hermite_reconstruct(lat, zero, torch.zeros_like(u), a2neq)  # a0_neq = a1_neq = 0
    return feq + (1.0 - omega).unsqueeze(0) * fneq + 0.5 * S


def shift_from(x, c):
    """Value of field x at site (position - c), periodic: out[r] = x[r - c].
    Field axes are (..., z, y, x); c = (cx, cy, cz)."""
    return torch.roll(x, shifts=(int(c[2]), int(c[1]), int(c[0])), dims=(-3, -2, -1))


def stream(lat, fpost, solid=None):
    """Pull streaming f_i(x) = f_post_i(x - c_i), periodic in every axis, with halfway
    bounce-back f_i(x) = f_post_opp(i)(x) where x - c_i is solid."""
    out = torch.empty_like(fpost)
    for i in range(lat.Q):
        ci = lat.ci[i]
        pulled = shift_from(fpost[i], ci)
        if solid is not None:
            src_solid = shift_from(solid, ci)
            pulled = torch.where(src_solid, fpost[lat.opp[i]], pulled)
        out[i] = pulled
    return out


def step(lat, f, F, rho, omega, solid=None):
    """One population-form time step (collide with the force at time t, then stream)."""
    return stream(lat, collide(lat, f, F, rho, omega), solid)


def omega_from_tau(tau):
    return 1.0 / torch.as_tensor(tau, dtype=torch.float64)


def viscosity(tau):
    """nu = cs2 (tau - 1/2) (text under Eq. pullLB)."""
    return CS2 * (tau - 0.5)


def run(lat, M0, steps, tau, force=(0.0, 0.0, 0.0), solid=None, rho=1.0, callback=None):
    """Single-component run from the public moment state M0 for `steps` steps.

    force: uniform 3-vector or per-site field (3, nz, ny, nx), constant in time.
    solid: bool (nz, ny, nx) or None; solid sites keep their input moments.
    callback(t, M) is called with the moment state after each step (t = 1..steps).
    Returns the public moment state after `steps` steps (FP64).
    """
    M0 = torch.as_tensor(M0, dtype=torch.float64)
    shape = M0.shape[1:]
    F = as_field(force, shape)
    rho_f = as_scalar_field(rho, shape)
    omega = as_scalar_field(omega_from_tau(tau), shape)
    if solid is not None:
        solid = torch.as_tensor(solid, dtype=torch.bool)
    f = populations_from_moments(lat, M0, F, rho_f)
    M = M0
    for t in range(1, steps + 1):
        f = step(lat, f, F, rho_f, omega, solid)
        if callback is not None or t == steps:
            M = moments_from_populations(lat, f, F, rho_f)
            if solid is not None:
                M = torch.where(solid.unsqueeze(0), M0, M)
            if callback is not None:
                callback(t, M)
    return M


def step_moments(lat, M, tau, force_src=(0.0, 0.0, 0.0), force_dst=None, solid=None,
                 rho_src=1.0, rho_dst=None):
    """One step as a map between public moment states, through explicit populations.
    force_src/rho_src are taken at time t (sources), force_dst/rho_dst at t+1 (Eq. corr)."""
    M = torch.as_tensor(M, dtype=torch.float64)
    shape = M.shape[1:]
    Fs = as_field(force_src, shape)
    Fd = Fs if force_dst is None else as_field(force_dst, shape)
    rs = as_scalar_field(rho_src, shape)
    rd = rs if rho_dst is None else as_scalar_field(rho_dst, shape)
    omega = as_scalar_field(omega_from_tau(tau), shape)
    if solid is not None:
        solid = torch.as_tensor(solid, dtype=torch.bool)
    f = populations_from_moments(lat, M, Fs, rs)
    f = step(lat, f, Fs, rs, omega, solid)
    out = moments_from_populations(lat, f, Fd, rd)
    if solid is not None:
        out = torch.where(solid.unsqueeze(0), M, out)
    return out


def step_at_sites(lat, M, sites, tau, force=(0.0, 0.0, 0.0), solid=None, rho=1.0):
    """One step evaluated only at the listed sites (z, y, x) of a possibly large state M,
    from the moments of their Q source neighbours. Same arithmetic as step_moments, restricted
    to a gathered neighbourhood; used to check full-size runs site by site.
    force: uniform 3-vector or field (3, nz, ny, nx). Returns (10, S) FP64."""
    M = torch.as_tensor(M, dtype=torch.float64)
    nz, ny, nx = M.shape[1:]
    sites = torch.as_tensor(sites, dtype=torch.int64).reshape(-1, 3)
    S = sites.shape[0]
    field_force = torch.as_tensor(force, dtype=torch.float64).dim() > 1
    omega = omega_from_tau(tau)

    def gather(field, z, y, x):
        return field[..., z, y, x]

    def force_at(z, y, x):
        if field_force:
            return gather(torch.as_tensor(force, dtype=torch.float64), z, y, x)
        return as_field(force, (S,))

    def post_all_directions(z, y, x):
        """f_post (Q, S) at the given sites from their own moments."""
        Ms = gather(M, z, y, x).unsqueeze(-1)  # (10, S, 1): a tiny one-site-per-row field
        Fs = force_at(z, y, x).unsqueeze(-1)
        rho_s = as_scalar_field(rho, (S, 1))
        om = as_scalar_field(omega, (S, 1))
        f = populations_from_moments(lat, Ms, Fs, rho_s)
        return collide(lat, f, Fs, rho_s, om)[..., 0]

    z0, y0, x0 = sites[:, 0], sites[:, 1], sites[:, 2]
    own_post = post_all_directions(z0, y0, x0)
    f_in = torch.empty((lat.Q, S), dtype=torch.float64)
    for i in range(lat.Q):
        cx, cy, cz = (int(v) for v in lat.ci[i])
        zs, ys, xs = (z0 - cz) % nz, (y0 - cy) % ny, (x0 - cx) % nx
        src_post = post_all_directions(zs, ys, xs)[i]
        if solid is not None:
            sol = torch.as_tensor(solid, dtype=torch.bool)[zs, ys, xs]
            src_post = torch.where(sol, own_post[lat.opp[i]], src_post)
        f_in[i] = src_post
    Fx = force_at(z0, y0, x0)
    out = moments_from_populations(lat, f_in, Fx, as_scalar_field(rho, (S,)))
    if solid is not None:
        own_solid = torch.as_tensor(solid, dtype=torch.bool)[z0, y0, x0]
        out = torch.where(own_solid.unsqueeze(0), gather(M, z0, y0, x0), out)
    return out
