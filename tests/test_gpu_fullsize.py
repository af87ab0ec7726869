"""Full-size checks in the benchmark's launch configuration: the 256^3 D3Q19 channel (FP32; the row
split of the library, also on a 512^3 channel) and the 512^3 D3Q27 Taylor-Green (FP32 and FP16 storage). The oracle recomputes one step at sampled
sites - at random, next to the walls and on CTA tile seams - from the GPU's own state before
that step; properties that hold at any size (mass conservation) are checked on the whole box."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import lbm

from paper_2609_09160_gb300 import Solver

from _helpers import group_errors

pytestmark = pytest.mark.gpu
LAT = {19: oracle.D3Q19, 27: oracle.D3Q27}


def neighbourhoods(M, sites, mask=None, field=None):
    """3x3x3 blocks around each site laid side by side along x: (.., 3, 3, 3S). On this small
    periodic lattice the centre column of each block sees exactly its true neighbours."""
    nz, ny, nx = M.shape[1:]
    S = sites.shape[0]
    off = torch.arange(-1, 2, device=M.device)
    z = (sites[:, 0, None] + off[None, :]) % nz  # (S, 3)
    y = (sites[:, 1, None] + off[None, :]) % ny
    x = (sites[:, 2, None] + off[None, :]) % nx
    zz = z[:, :, None, None].expand(S, 3, 3, 3)
    yy = y[:, None, :, None].expand(S, 3, 3, 3)
    xx = x[:, None, None, :].expand(S, 3, 3, 3)

    def block(t):
        b = t[..., zz, yy, xx]  # (..., S, 3, 3, 3)
        b = b.movedim(-4, -2)  # (..., 3, 3, S, 3)
        return b.reshape(b.shape[:-2] + (3 * S,)).cpu()
    return block(M), (None if mask is None else block(mask)), (None if field is None else block(field))


def sample_sites(shape, n, seed, extra=()):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    pts = np.stack([rng.integers(0, nz, n), rng.integers(0, ny, n), rng.integers(0, nx, n)], 1)
    pts = np.concatenate([pts, np.array(list(extra), dtype=np.int64).reshape(-1, 3)], 0)
    return torch.from_numpy(pts)


def check_one_step(s, lat, tau, force, sites, mask=None, tol=1e-5):
    before = s.moments()  # FP64 decode of the state the GPU holds
    s.step(1)
    after = s.moments()
    sd = sites.to(before.device)
    Mb, mb, _ = neighbourhoods(before, sd, None if mask is None else mask.to(before.device))
    want = lbm.step_moments(lat, Mb, tau, torch.tensor(force, dtype=torch.float64), solid=mb)
    want = want[:, 1, 1, 1::3]
    got = after[:, sd[:, 0], sd[:, 1], sd[:, 2]].cpu()
    err = group_errors(got, want)
    assert max(err.values()) < tol, err


def test_channel_256_d3q19_fp32_sampled():
    shape = (256, 256, 256)
    M0, solid = synth.channel(shape, 1e-3, seed=1)
    s = Solver(shape, lattice=19, tau=0.9, storage="f32", force=(1e-6, 0.0, 0.0), mask=solid)
    s.set_moments(M0.to(torch.float32).cuda())
    r0 = s.reduce()
    s.step(20)
    # 30-column tile seams (masked kernel), the row split's boundaries (rows 249 | 250 and 1 | 2: the
    # periodic line-aligned kernel runs rows 2..249), its 32 x 8 tile seams and z-chunk seams
    seams = [(7, 1, 0), (7, 1, 29), (7, 1, 30), (8, 254, 255), (100, 8, 59), (100, 9, 60), (255, 255, 17),
             (0, 128, 240), (63, 64, 241), (64, 65, 239), (21, 249, 31), (22, 250, 32), (43, 1, 63), (44, 2, 64),
             (0, 9, 95), (100, 10, 96), (255, 253, 128), (128, 254, 31), (21, 2, 255), (22, 249, 0)]
    check_one_step(s, LAT[19], 0.9, (1e-6, 0.0, 0.0), sample_sites(shape, 3000, 2, seams), solid)
    r1 = s.reduce()
    assert abs(r1[0] - r0[0]) < 1e-6 * M0[0].abs().sum().item()
    assert r1[1] > 0  # the body force accelerates the fluid along +x


def test_channel_512_d3q19_fp32_sampled():
    """The row split on a 512^3 channel: rows 2..505 on the periodic line-aligned kernel, rows
    506..511, 0, 1 on the masked kernel beside it."""
    shape = (512, 512, 512)
    M0, solid = synth.channel(shape, 1e-3, seed=5)
    s = Solver(shape, lattice=19, tau=0.9, storage="f32", force=(1e-6, 0.0, 0.0), mask=solid)
    s.set_moments(M0.to(torch.float32).cuda())
    del M0
    s.step(3)
    seams = [(63, 505, 31), (64, 506, 32), (0, 1, 511), (511, 2, 0), (300, 9, 63), (301, 10, 64), (5, 510, 200)]
    check_one_step(s, LAT[19], 0.9, (1e-6, 0.0, 0.0), sample_sites(shape, 2000, 6, seams), solid)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 2e-3)])
def test_taylor_green_512_d3q27_sampled(storage, tol):
    n = 512
    M0 = synth.taylor_green_perturbed(n, 0.04, 0.55, 0.01, seed=3, dtype=torch.float32, device="cuda")
    s = Solver((n, n, n), lattice=27, tau=0.55, storage=storage)
    s.set_moments(M0)
    del M0
    s.step(5)
    seams = [(0, 0, 0), (511, 511, 511), (200, 7, 29), (200, 8, 30), (3, 511, 509)]
    check_one_step(s, LAT[27], 0.55, (0.0, 0.0, 0.0), sample_sites((n, n, n), 2000, 4, seams), tol=tol)
