"""Discrete velocity sets D3Q19 and D3Q27 (FP64), written out from their textbook definition.

The paper uses the standard D3Q19 and D3Q27 quadratures (Sec. 2, "D3Q19 and D3Q27 models
with the Hermite expansion truncated at second order") without printing the tables; the
values here are the textbook ones (Kruger et al., "The Lattice Boltzmann Method", Sec. 3.4):

    c_s^2 = 1/3
    D3Q19: rest 1/3, 6 face neighbours 1/18, 12 edge neighbours 1/36
    D3Q27: rest 8/27, 6 faces 2/27, 12 edges 1/54, 8 corners 1/216

The set is enumerated from {-1,0,1}^3 and the weight is a function of |c|^2 only. D3Q27H is
the D3Q27 set used with its complete Hermite basis (below).
The tests pin these tables by the isotropy identities of the quadrature, not by re-reading them.
"""
import itertools
import math

import torch

CS2 = 1.0 / 3.0  # lattice speed of sound squared

_WEIGHT_BY_NORM2 = {
    "D3Q19": {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0},
    "D3Q27": {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0},
}


# D3Q27h (Sec. 2: "a higher-order D3Q27h formulation based on the complete Hermite basis"): the
# D3Q27 velocities with every Hermite polynomial the lattice supports. On D3Q27 these are the 27
# products H_m(c) = h_mx(c_x) h_my(c_y) h_mz(c_z), m in {0,1,2}^3, of the one-dimensional
# polynomials h_0 = 1, h_1 = c, h_2 = c^2 - c_s^2 (the multi-index m counts how often each axis
# occurs in the tensor index, e.g. H_xxy = (c_x^2 - c_s^2) c_y); they are orthogonal under the
# D3Q27 weights with norms prod_a m_a! c_s^(2 m_a).
MULTI = tuple((mx, my, mz) for mz in range(3) for my in range(3) for mx in range(3))


def _h1d(m, c):
    return torch.ones_like(c) if m == 0 else (c if m == 1 else c * c - CS2)


def axes_of(m):
    """Tensor index tuple of multi-index m, e.g. (2, 1, 0) -> (0, 0, 1) (x, x, y)."""
    return tuple(a for a in range(3) for _ in range(m[a]))


class Lattice:
    """Velocity set: c (Q,3) in (x,y,z) order, w (Q,), opp (Q,) index of -c_i.
    high: the complete Hermite basis (D3Q27h) is used for the post-collision populations."""

    def __init__(self, name):
        self.high = name == "D3Q27H"
        table_name = "D3Q27" if self.high else name
        if table_name not in _WEIGHT_BY_NORM2:
            raise ValueError(f"unknown lattice {name!r}")
        table = _WEIGHT_BY_NORM2[table_name]
        vel, wts = [], []
        for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3):
            n2 = cx * cx + cy * cy + cz * cz
            if n2 in table:
                vel.append((cx, cy, cz))
                wts.append(table[n2])
        self.name = name
        self.Q = len(vel)
        self.c = torch.tensor(vel, dtype=torch.float64)
        self.ci = torch.tensor(vel, dtype=torch.int64)
        self.w = torch.tensor(wts, dtype=torch.float64)
        index = {v: i for i, v in enumerate(vel)}
        self.opp = torch.tensor([index[(-a, -b, -d)] for (a, b, d) in vel], dtype=torch.int64)
        eye = torch.eye(3, dtype=torch.float64)
        # second-order Hermite polynomial H2_i = c_i c_i - c_s^2 delta (Sec. 2, discrete Hermite basis)
        self.H2 = torch.einsum("qa,qb->qab", self.c, self.c) - CS2 * eye
        if table_name == "D3Q27":
            # full Hermite basis: HM (27, Q) and its norms (27,), rows in MULTI order
            self.HM = torch.stack([_h1d(m[0], self.c[:, 0]) * _h1d(m[1], self.c[:, 1]) * _h1d(m[2], self.c[:, 2])
                                   for m in MULTI])
            self.HM_norm = torch.tensor([math.prod(math.factorial(k) * CS2 ** k for k in m) for m in MULTI],
                                        dtype=torch.float64)

    def __repr__(self):
        return f"Lattice({self.name}, Q={self.Q})"


D3Q19 = Lattice("D3Q19")
D3Q27 = Lattice("D3Q27")
D3Q27H = Lattice("D3Q27H")


def get(name):
    return {"D3Q19": D3Q19, "D3Q27": D3Q27, "D3Q27H": D3Q27H}[name]
