"""The line-aligned fused kernel (32-column tiles, TMA tensor stores; FP32 and 16-bit storage, single
component) against the 30-column kernel (LBF_KERNEL=aligned / cta select them at lbf_create) and against the
oracle, on shapes that exercise partial tiles in x and y, the periodic wrap of the halo rows and
columns, walls and force fields. Both kernels evaluate the same expressions in the same order; the
compiler contracts a few of them into FMAs differently, so the states agree to a few units in the
last place of the storage type, not bit for bit."""
import os

import pytest
import torch

import oracle
import synth
from paper_2609_09160_gb300 import Solver

from _helpers import TOL, as_f32_exact, group_errors

pytestmark = pytest.mark.gpu
LAT = {19: oracle.D3Q19, 27: oracle.D3Q27}


def _solver(no_aligned, **kw):
    old = os.environ.pop("LBF_KERNEL", None)
    try:
        os.environ["LBF_KERNEL"] = "cta" if no_aligned else "aligned"
        return Solver(**kw)
    finally:
        os.environ.pop("LBF_KERNEL", None)
        if old is not None:
            os.environ["LBF_KERNEL"] = old


SHAPES = [(5, 13, 64), (7, 9, 40), (3, 17, 96), (9, 6, 32)]
# a few units in the last place of the stored value, relative to the largest value of a field group
ULPS = {"f32": 4 * 2.0 ** -23, "f16": 4 * 2.0 ** -10, "bf16": 4 * 2.0 ** -7}


@pytest.mark.parametrize("lattice", [19, 27, 127])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("kind", ["periodic", "walls", "field"])
def test_aligned_kernel_matches_30_column_kernel(lattice, storage, kind):
    for shape in SHAPES:
        M0 = synth.random_moments(shape, seed=40)
        kw = dict(shape=shape, lattice=lattice, tau=0.7, storage=storage, force=(1e-5, -2e-5, 3e-6))
        if kind == "walls":
            kw["mask"] = synth.channel_walls(shape) | synth.random_mask(shape, 0.05, seed=41)
        if kind == "field":
            kw["force_field"] = synth.random_field(shape, 1e-4, seed=42).to(device="cuda", dtype=torch.float32)
        a = _solver(False, **kw)
        b = _solver(True, **kw)
        for s in (a, b):
            s.set_moments(M0.cuda())
            s.step(3)
        err = group_errors(a.moments(), b.moments())
        assert max(err.values()) < ULPS[storage], (shape, err)
        # the sums add the computed values; in 16-bit storage the states they come from differ by
        # the rounding of a few values, so the bound scales with the sum of magnitudes
        ra, rb = a.reduce(), b.reduce()
        mag = [M0[0].abs().sum().item()] + [M0[1 + i].abs().sum().item() for i in range(3)]
        mag += [1.0, (M0[1:4] ** 2).sum().item()]
        for k in (0, 1, 2, 3, 5):
            assert abs(ra[k] - rb[k]) <= ULPS[storage] * max(1.0, mag[k]), (k, ra[k], rb[k])


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("kind", ["periodic", "walls"])
def test_aligned_kernel_matches_oracle(lattice, kind):
    shape = (6, 14, 40)  # partial x tile (40 = 32 + 8) and partial y tiles
    M0 = synth.random_moments(shape, seed=43)
    mask = (synth.channel_walls(shape) | synth.random_mask(shape, 0.05, seed=44)) if kind == "walls" else None
    s = _solver(False, shape=shape, lattice=lattice, tau=0.8, storage="f32", force=(2e-5, 0.0, -1e-5), mask=mask)
    s.set_moments(M0.cuda())
    s.step(4)
    want = oracle.lbm.run(LAT[lattice], as_f32_exact(M0), 4, 0.8, force=(2e-5, 0.0, -1e-5), solid=mask)
    err = group_errors(s.moments(), want)
    assert max(err.values()) < TOL["f32"], err
