"""Walls confined to a band of rows: the library splits a step into the rows clear of every solid
site and of its neighbours (the periodic line-aligned kernel, no mask logic) and the remaining rows
(the masked 30-column kernel, on a side stream), and adds both launches' partial sums in one more
kernel. LBF_KERNEL=split selects the split on any plane size, LBF_KERNEL=cta the single masked
launch. The split must give the state of the single launch to a few units in the last place (the
two kernels round a few multiply-adds differently), the sums of the fluid sites, and the oracle's
state within the FP32 parity tolerance; solid sites keep their stored state."""
import os

import pytest
import torch

import oracle
import synth
from paper_2609_09160_gb300 import Solver

from _helpers import TOL, as_f32_exact, group_errors

pytestmark = pytest.mark.gpu
LAT = {19: oracle.D3Q19, 27: oracle.D3Q27}
ULPS_F32 = 4 * 2.0 ** -23


def _solver(kernel, **kw):
    old = os.environ.pop("LBF_KERNEL", None)
    try:
        os.environ["LBF_KERNEL"] = kernel
        return Solver(**kw)
    finally:
        os.environ.pop("LBF_KERNEL", None)
        if old is not None:
            os.environ["LBF_KERNEL"] = old


def _walls(shape, rows):
    m = torch.zeros(shape, dtype=torch.bool)
    for y in rows:
        m[:, y, :] = True
    return m


# (shape (nz, ny, nx), solid rows): channel walls at both ends, a wall in the middle (two clean
# runs: the longer one is split off), a run that wraps around y = 0, a partial wall row, and ragged
# x and y tiles
CASES = [((5, 30, 64), (0, 29)), ((3, 41, 40), (20,)), ((4, 26, 96), (9, 10)), ((2, 33, 36), (0,)),
         ((6, 28, 64), "partial")]


def _mask(shape, rows):
    if rows == "partial":  # solids in rows 0 and 1 over a third of x only
        m = torch.zeros(shape, dtype=torch.bool)
        m[:, 0:2, : shape[2] // 3] = True
        return m
    return _walls(shape, rows)


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_split_step_matches_single_masked_launch(lattice, case):
    shape, rows = CASES[case]
    mask = _mask(shape, rows)
    M0 = synth.random_moments(shape, seed=50 + case)
    kw = dict(shape=shape, lattice=lattice, tau=0.7, storage="f32", force=(1e-5, -2e-6, 3e-6), mask=mask)
    a = _solver("split", **kw)
    b = _solver("cta", **kw)
    for s in (a, b):
        s.set_moments(M0.cuda())
        s.step(4)
    err = group_errors(a.moments(), b.moments())
    assert max(err.values()) < ULPS_F32, (shape, rows, err)
    ra, rb = a.reduce(), b.reduce()
    fluid = ~mask
    mag = [M0[0][fluid].abs().sum().item()] + [M0[1 + i][fluid].abs().sum().item() for i in range(3)]
    mag += [1.0, (M0[1:4][:, fluid] ** 2).sum().item()]
    for k in (0, 1, 2, 3, 5):
        assert abs(ra[k] - rb[k]) <= 8 * ULPS_F32 * max(1.0, mag[k]), (k, ra[k], rb[k])
    # solid sites keep their stored state
    sa, sb = a.new_state(), b.new_state()
    a.copy_state(sa)
    b.copy_state(sb)
    va = sa.view(torch.float32).reshape((10,) + shape).cpu()
    vb = sb.view(torch.float32).reshape((10,) + shape).cpu()
    assert (va[:, mask] == vb[:, mask]).all()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_split_step_16bit_matches_single_masked_launch(storage):
    """16-bit storage (D3Q19): both kernels draw the same stochastic-rounding words (keyed by site
    and step), so the states differ only where the FP32 values before rounding differ in their last
    bits: by at most a few units of the 16-bit format, at few sites."""
    ulps = {"f16": 4 * 2.0 ** -10, "bf16": 4 * 2.0 ** -7}[storage]
    for case in (0, 1, 4):
        shape, rows = CASES[case]
        mask = _mask(shape, rows)
        M0 = synth.random_moments(shape, seed=60 + case)
        kw = dict(shape=shape, lattice=19, tau=0.7, storage=storage, force=(1e-5, -2e-6, 3e-6), mask=mask)
        a = _solver("split", **kw)
        b = _solver("cta", **kw)
        for s in (a, b):
            s.set_moments(M0.cuda())
            s.step(3)
        err = group_errors(a.moments(), b.moments())
        assert max(err.values()) < ulps, (shape, rows, err)


@pytest.mark.parametrize("lattice", [19, 27])
def test_split_step_matches_oracle(lattice):
    shape = (5, 30, 64)
    mask = _walls(shape, (0, 29))
    M0 = synth.random_moments(shape, seed=57)
    s = _solver("split", shape=shape, lattice=lattice, tau=0.8, storage="f32", force=(2e-5, 0.0, -1e-5), mask=mask)
    s.set_moments(M0.cuda())
    s.step(4)
    want = oracle.lbm.run(LAT[lattice], as_f32_exact(M0), 4, 0.8, force=(2e-5, 0.0, -1e-5), solid=mask)
    err = group_errors(s.moments(), want)
    assert max(err.values()) < TOL["f32"], err


def test_split_sums_and_state_deterministic_and_step_state_unsplit():
    """Two runs of the split step give the same bits (sums included); a step between caller buffers
    (lbf_step_state, which the split does not cover) gives the same state to rounding."""
    shape = (4, 30, 64)
    mask = _walls(shape, (0, 29))
    M0 = synth.random_moments(shape, seed=58)
    outs = []
    for _ in range(2):
        s = _solver("split", shape=shape, lattice=19, tau=0.75, storage="f32", force=(1e-5, 0.0, 0.0), mask=mask)
        s.set_moments(M0.cuda())
        s.step(3)
        outs.append((s.moments().cpu(), s.reduce()))
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    s = _solver("split", shape=shape, lattice=19, tau=0.75, storage="f32", force=(1e-5, 0.0, 0.0), mask=mask)
    s.set_moments(M0.cuda())
    x = s.new_state()
    s.copy_state(x)
    y = s.new_state()
    s.copy_state(y)  # a step does not write solid sites: dst starts as a copy
    s.step_state(x, y)
    s.load_state(y)
    t = _solver("split", shape=shape, lattice=19, tau=0.75, storage="f32", force=(1e-5, 0.0, 0.0), mask=mask)
    t.set_moments(M0.cuda())
    t.step(1)
    err = group_errors(s.moments(), t.moments())
    assert max(err.values()) < ULPS_F32, err
