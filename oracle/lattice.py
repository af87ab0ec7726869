"""Discrete velocity sets D3Q19 and D3Q27 (FP64), written out from their textbook definition.

The paper uses the standard D3Q19 and D3Q27 quadratures (Sec. 2, "D3Q19 and D3Q27 models
with the Hermite expansion truncated at second order") without printing the tables; the
values here are the textbook ones (Kruger et al., "The Lattice Boltzmann Method", Sec. 3.4):

    c_s^2 = 1/3
    D3Q19: rest 1/3, 6 face neighbours 1/18, 12 edge neighbours 1/36
    D3Q27: rest 8/27, 6 faces 2/27, 12 edges 1/54, 8 corners 1/216

The set is enumerated from {-1,0,1}^3 and the weight is a function of |c|^2 only.
The tests pin these tables by the isotropy identities of the quadrature, not by re-reading them.
"""
import itertools

import torch

CS2 = 1.0 / 3.0  # lattice speed of sound squared

_WEIGHT_BY_NORM2 = {
    "D3Q19": {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0},
    "D3Q27": {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0},
}


class Lattice:
    """Velocity set: c (Q,3) in (x,y,z) order, w (Q,), opp (Q,) index of -c_i."""

    def __init__(self, name):
        if name not in _WEIGHT_BY_NORM2:
            raise ValueError(f"unknown lattice {name!r}")
        table = _WEIGHT_BY_NORM2[name]
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

    def __repr__(self):
        return f"Lattice({self.name}, Q={self.Q})"


D3Q19 = Lattice("D3Q19")
D3Q27 = Lattice("D3Q27")


def get(name):
    return {"D3Q19": D3Q19, "D3Q27": D3Q27}[name]
