"""lbf_step_static: the step entry point for callers that cannot allocate device memory.

Code running under another framework's memory pool, under a fixed memory plan, or embedded where
it only receives device buffers, cannot call cudaMalloc and so cannot hand lbf_create a workspace.
lbf_step_static takes only the caller's state buffers (and optional mask, sums and flags outputs)
and keeps its reduction scratch in a static device array inside the library. Here two calls in a
row of it, through the C ABI, must reproduce two steps of the context-based entry point
(lbf_step_state) within the parity tolerance of the other tests, including the conservation sums,
for every lattice with and without walls; the flags word must reach the caller.

This file is named to be collected last.
"""
import pytest
import torch

import synth
from paper_2609_09160_gb300 import LBFError, Solver, _lbf

from _helpers import TOL, group_errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lattice", [19, 27, 127])
@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("nx", [64, 37])
@pytest.mark.parametrize("walls", [True, False])
def test_static_scratch_step_matches_context_step(lattice, storage, nx, walls):
    shape = (20, 26, nx)  # several z-chunks and y-tiles; nx = 64 stages planes with TMA, 37 loads directly
    M0 = synth.random_moments(shape, seed=90)
    mask = (synth.channel_walls(shape) | synth.random_mask(shape, 0.05, seed=91)) if walls else None
    s = Solver(shape, lattice=lattice, tau=0.7, storage=storage, force=(1e-5, 0.0, -2e-5), mask=mask)
    s.set_moments(M0.cuda())
    x0 = s.new_state()
    s.copy_state(x0)

    # two steps through the existing, context-based entry point
    r1, r2 = x0.clone(), x0.clone()  # solid sites are not written by a step
    s.step_state(x0, r1)
    s.step_state(r1, r2)

    # two calls in a row of the no-allocation entry point, same parameters (device mask, if any)
    p = _lbf.lbf_params.from_buffer_copy(s.params)
    p.mask = None
    mask_d = mask.to(device="cuda", dtype=torch.uint8).contiguous() if walls else None
    mask_ptr = mask_d.data_ptr() if walls else None
    sums = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    flags = torch.full((2,), 0x7777, dtype=torch.int32, device="cuda")
    y1, y2 = x0.clone(), x0.clone()
    _lbf.lbf_step_static(p, x0.data_ptr(), y1.data_ptr(), mask_ptr, sums.data_ptr(), flags.data_ptr())
    _lbf.lbf_step_static(p, y1.data_ptr(), y2.data_ptr(), mask_ptr, sums.data_ptr(), flags[1:].data_ptr())
    torch.cuda.synchronize()
    assert flags.tolist() == [0, 0]  # both steps completed, stable

    for got_state, ref_state in ((y1, r1), (y2, r2)):
        s.load_state(ref_state)
        ref = s.moments()
        s.load_state(got_state)
        got = s.moments()
        err = group_errors(got, ref)
        assert max(err.values()) < TOL[storage], err

    s.load_state(r2)
    ref_sums = s.reduce()
    got_sums = sums.cpu().tolist()
    tol = 1e-12 if storage == "f64" else 1e-6
    scale = [abs(M0[0]).sum().item(), *(abs(M0[1 + a]).sum().item() for a in range(3)), 1.0,
             (M0[1:4] ** 2).sum().item()]
    for k in (0, 1, 2, 3, 5):
        assert abs(got_sums[k] - ref_sums[k]) <= tol * scale[k], (k, got_sums[k], ref_sums[k])


@pytest.mark.parametrize("lattice", [19, 27])
def test_static_scratch_without_sums_or_alignment(lattice):
    """No sums output (no reduction runs) and a state that is not 16-byte aligned (a view one FP32
    element into a larger buffer: the direct-load kernel instead of TMA) give the same step."""
    shape = (9, 14, 64)
    M0 = synth.random_moments(shape, seed=92)
    s = Solver(shape, lattice=lattice, tau=0.75, storage="f32", force=(0.0, 3e-5, 0.0))
    s.set_moments(M0.cuda())
    x0 = s.new_state()
    s.copy_state(x0)
    r1 = x0.clone()
    s.step_state(x0, r1)
    p = _lbf.lbf_params.from_buffer_copy(s.params)
    nb = x0.numel()
    src = torch.empty(nb + 4, dtype=torch.uint8, device="cuda")
    src[4:].copy_(x0)
    y1 = x0.clone()
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    _lbf.lbf_step_static(p, src[4:].data_ptr(), y1.data_ptr(), None, None, flags.data_ptr())
    torch.cuda.synchronize()
    assert flags.item() == 0
    s.load_state(r1)
    ref = s.moments()
    s.load_state(y1)
    got = s.moments()
    err = group_errors(got, ref)
    assert max(err.values()) < TOL["f32"], err


def test_static_scratch_reports_instability():
    """A state with |u| above the stability bound sets bit 0 of the caller's flags word."""
    shape = (4, 8, 32)
    M0 = synth.random_moments(shape, seed=93)
    M0[1] += 0.6
    s = Solver(shape, lattice=19, tau=0.8, storage="f32")
    s.set_moments(M0.cuda())
    x0 = s.new_state()
    s.copy_state(x0)
    y = x0.clone()
    p = _lbf.lbf_params.from_buffer_copy(s.params)
    flags = torch.zeros((1,), dtype=torch.int32, device="cuda")
    _lbf.lbf_step_static(p, x0.data_ptr(), y.data_ptr(), None, None, flags.data_ptr())
    torch.cuda.synchronize()
    assert flags.item() == 1


def test_static_scratch_rejects_lattices_beyond_its_capacity():
    p = _lbf.lbf_params()
    p.lattice, p.nx, p.ny, p.nz, p.storage, p.tau = 19, 30 * 16385, 8, 1, _lbf.LBF_F32, 0.8
    buf = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(LBFError) as e:
        _lbf.lbf_step_static(p, buf.data_ptr(), buf[8:].data_ptr())
    assert e.value.status == _lbf.LBF_EINVAL
    assert "16384" in str(e.value)
