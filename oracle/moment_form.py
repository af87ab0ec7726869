"""Literal, site-by-site transcription of the moment-represented update, Eq. (pullLLB) + Eq. (corr).

TEST INFRASTRUCTURE (oracle). Pure-Python loops: meant for tiny lattices (4^3), where it is
compared with the population form in oracle.lbm to show that the two formulations agree.

For each site x and each direction i, the bracket of Eq. (pullLLB) is evaluated at the source
x - c_i and time t:

    B_i = w_i sum_{m=0..2} H^(m)_i : (a_eq^(m) + (1 - omega) a_neq^(m)) / (cs2^m m!) + S_i / 2

with a_eq = (p*, u, u u) and a_neq = (0, 0, A - u u) (velocity form, Sec. 2). The new Hermite
coefficients are a*^(n)(x) = sum_i H^(n)_i B_i, then Eq. (corr) adds the half-force shift with
the force at x and t+1. Where x - c_i is solid, the bracket of the opposite direction is taken
at x itself (halfway bounce-back).
"""
from .lattice import CS2
from .lbm import SYM


def _bracket(lat, i, Ms, Fs, rho, omega):
    """B_i of Eq. (pullLLB) from the 10 public moments Ms at one source site."""
    p = Ms[0]
    u = Ms[1:4]
    A = [[0.0] * 3 for _ in range(3)]
    for k, (a, b) in enumerate(SYM):
        A[a][b] = Ms[4 + k]
        A[b][a] = Ms[4 + k]
    c = [float(v) for v in lat.c[i]]
    w = float(lat.w[i])
    H2 = [[c[a] * c[b] - (CS2 if a == b else 0.0) for b in range(3)] for a in range(3)]
    m0 = p  # H^(0) = 1, a_neq^(0) = 0
    m1 = sum(c[a] * u[a] for a in range(3)) / CS2  # a_neq^(1) = 0
    m2 = 0.0
    for a in range(3):
        for b in range(3):
            aeq = u[a] * u[b]
            aneq = A[a][b] - u[a] * u[b]
            m2 += H2[a][b] * (aeq + (1.0 - omega) * aneq)
    m2 /= 2.0 * CS2 * CS2
    cu = sum(c[a] * u[a] for a in range(3))
    S = w * sum(((c[a] - u[a]) / CS2 + cu * c[a] / (CS2 * CS2)) * Fs[a] for a in range(3)) / rho
    return w * (m0 + m1 + m2) + 0.5 * S


def step(lat, M, tau, force_src, force_dst, solid=None, rho=1.0):
    """One step on nested Python lists. M: [10][nz][ny][nx]; force_*: [3][nz][ny][nx];
    solid: [nz][ny][nx] of bool or None. Returns the new [10][nz][ny][nx]."""
    nz, ny, nx = len(M[0]), len(M[0][0]), len(M[0][0][0])
    omega = 1.0 / tau
    out = [[[[M[k][z][y][x] for x in range(nx)] for y in range(ny)] for z in range(nz)] for k in range(10)]

    def at(field, ncomp, z, y, x):
        return [field[k][z][y][x] for k in range(ncomp)]

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if solid is not None and solid[z][y][x]:
                    continue
                a0 = 0.0
                a1 = [0.0, 0.0, 0.0]
                a2 = [[0.0] * 3 for _ in range(3)]
                for i in range(lat.Q):
                    cx, cy, cz = (int(v) for v in lat.ci[i])
                    zs, ys, xs = (z - cz) % nz, (y - cy) % ny, (x - cx) % nx
                    if solid is not None and solid[zs][ys][xs]:
                        B = _bracket(lat, int(lat.opp[i]), at(M, 10, z, y, x),
                                     at(force_src, 3, z, y, x), rho, omega)
                    else:
                        B = _bracket(lat, i, at(M, 10, zs, ys, xs), at(force_src, 3, zs, ys, xs),
                                     rho, omega)
                    c = [float(v) for v in lat.c[i]]
                    a0 += B
                    for a in range(3):
                        a1[a] += c[a] * B
                        for b in range(3):
                            a2[a][b] += (c[a] * c[b] - (CS2 if a == b else 0.0)) * B
                F = at(force_dst, 3, z, y, x)
                u = [a1[a] + F[a] / (2.0 * rho) for a in range(3)]  # Eq. (corr)
                A = [[a2[a][b] + (F[a] * u[b] + F[b] * u[a]) / (2.0 * rho) for b in range(3)]
                     for a in range(3)]
                out[0][z][y][x] = a0
                for a in range(3):
                    out[1 + a][z][y][x] = u[a]
                for k, (a, b) in enumerate(SYM):
                    out[4 + k][z][y][x] = A[a][b]
    return out
