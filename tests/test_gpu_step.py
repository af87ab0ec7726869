"""GPU parity of the fused step (through the C ABI) with the FP64 oracle: element by element on
seeded inputs spanning several CTA tiles with ragged tails, every lattice x storage x boundary
and force combination, degenerate boxes, 16-bit storage error bounds, conservation sums and the
host-memory transfer paths."""
import pytest
import torch

import oracle
import synth
from oracle import diagnostics as dg
from oracle import lbm
from paper_2609_09160_gb300 import LBFError, Solver

from _helpers import TOL, group_errors, rel_max

pytestmark = pytest.mark.gpu
LAT = {19: oracle.D3Q19, 27: oracle.D3Q27}
CDT = {"f64": torch.float64, "f32": torch.float32}


def make_case(case, shape, storage, seed=0):
    M0 = synth.random_moments(shape, seed=seed)
    force = (0.0, 0.0, 0.0)
    field = None
    mask = None
    if case == "uniform_force":
        force = (2e-5, -1e-5, 5e-6)
    if case == "walls_field":
        mask = synth.channel_walls(shape) | synth.random_mask(shape, 0.1, seed=seed + 1)
        field = synth.random_field(shape, 1e-4, seed=seed + 2, mask=mask)
        force = (1e-5, 0.0, 0.0)
    return M0, force, field, mask


def run_gpu(lattice, storage, shape, M0, force, field, mask, steps, tau):
    ff = None if field is None else field.to(device="cuda", dtype=CDT[storage]).contiguous()
    s = Solver(shape, lattice=lattice, tau=tau, storage=storage, force=force, force_field=ff, mask=mask)
    s.set_moments(M0.cuda())
    s.step(steps)
    return s.moments(), s


def run_oracle(lattice, storage, M0, force, field, mask, steps, tau):
    F = torch.tensor(force, dtype=torch.float64)
    if field is not None:
        F = F.reshape(3, 1, 1, 1) + field.to(CDT[storage]).to(torch.float64)
    return lbm.run(LAT[lattice], M0, steps, tau, force=F, solid=mask)


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case", ["periodic", "uniform_force", "walls_field"])
@pytest.mark.parametrize("nx", [37, 36])
def test_step_matches_oracle(lattice, storage, case, nx):
    """nx = 37: rows are not 16-byte multiples, planes load directly; nx = 36: TMA plane patches.
    2 x-tiles (30 wide), 2-4 y-tiles, 2 z-chunks, ragged everywhere."""
    shape = (11, 13, nx)
    M0, force, field, mask = make_case(case, shape, storage, seed=lattice)
    got, _ = run_gpu(lattice, storage, shape, M0, force, field, mask, 5, 0.7)
    want = run_oracle(lattice, storage, M0, force, field, mask, 5, 0.7)
    err = group_errors(got, want)
    assert max(err.values()) < TOL[storage], err


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 2), (2, 1, 5), (3, 4, 1), (5, 2, 31), (9, 17, 30),
                                   (1, 1, 2), (3, 5, 4), (2, 3, 8), (4, 9, 60), (3, 2, 62)])
def test_degenerate_and_tile_edge_shapes(lattice, shape):
    M0, force, field, mask = make_case("uniform_force", shape, "f64", seed=3)
    got, _ = run_gpu(lattice, "f64", shape, M0, force, None, None, 3, 0.9)
    want = run_oracle(lattice, "f64", M0, force, None, None, 3, 0.9)
    assert max(group_errors(got, want).values()) < TOL["f64"]


@pytest.mark.parametrize("lattice", [19, 27])
def test_single_wall_site_and_fully_solid_rows(lattice):
    shape = (4, 6, 33)
    M0 = synth.random_moments(shape, seed=8)
    mask = torch.zeros(shape, dtype=torch.bool)
    mask[2, 3, 17] = True
    mask[:, 0, :] = True
    got, _ = run_gpu(lattice, "f64", shape, M0, (0.0, 1e-5, 0.0), None, mask, 4, 0.75)
    want = run_oracle(lattice, "f64", M0, (0.0, 1e-5, 0.0), None, mask, 4, 0.75)
    assert max(group_errors(got, want).values()) < TOL["f64"]


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("storage,bound", [("f16", 5e-3), ("bf16", 4e-2)])
@pytest.mark.parametrize("nx", [34, 40])
def test_16bit_storage_error_against_fp64(lattice, storage, bound, nx):
    """16-bit deviation storage with FP32 arithmetic: the error of p*, u and A against the FP64
    oracle stays within the storage rounding accumulated over the steps (stated, not exact).
    nx = 40 takes the TMA path (80-byte rows), nx = 34 the direct loads."""
    shape = (10, 12, nx)
    M0 = synth.taylor_green_perturbed(shape, 0.04, 0.6, 0.01, seed=5)
    got, _ = run_gpu(lattice, storage, shape, M0, (0.0, 0.0, 0.0), None, None, 10, 0.6)
    want = run_oracle(lattice, "f64", M0, (0.0, 0.0, 0.0), None, None, 10, 0.6)
    err = group_errors(got, want)
    assert err["u"] < bound, err
    assert max(err.values()) < 10 * bound, err


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_conservation_sums(storage):
    shape = (12, 14, 40)
    M0 = synth.random_moments(shape, seed=21)
    s = Solver(shape, lattice=19, tau=0.65, storage=storage)
    s.set_moments(M0.cuda())
    r0 = s.reduce()
    ref0 = dg.reductions(M0)
    tol = 1e-12 if storage == "f64" else 1e-6
    scale_p = M0[0].abs().sum().item()
    scale_u = M0[1:4].abs().sum().item()
    assert abs(r0[0] - ref0[0].item()) < tol * scale_p
    s.step(10)
    r1 = s.reduce()
    assert abs(r1[0] - r0[0]) < tol * scale_p
    for a in range(3):
        assert abs(r1[1 + a] - r0[1 + a]) < tol * scale_u
    # sum u.u of the final state against the oracle's reduction of the GPU's own output
    ref1 = dg.reductions(s.moments().cpu())
    n = M0[0].numel()
    assert abs(r1[5] / 2 / n - ref1[5].item()) < 1e-5 * ref1[5].item()


def test_reduce_async_matches_reduce():
    """lbf_reduce_async copies, without waiting, the same FP64 sums lbf_reduce returns: one pinned
    host row per step collects the series, and a device buffer gets the latest ones."""
    shape = (6, 20, 32)
    M0 = synth.random_moments(shape, seed=47)
    kw = dict(lattice=19, tau=0.8, storage="f32", force=(1e-5, 0.0, 0.0), mask=synth.channel_walls(shape))
    a = Solver(shape, **kw)
    a.set_moments(M0.cuda())
    series = torch.empty((4, 6), dtype=torch.float64).pin_memory()
    dev = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    for k in range(4):
        a.step(1)
        a.reduce_async(series[k])
    a.reduce_async(dev)
    a.synchronize()
    b = Solver(shape, **kw)
    b.set_moments(M0.cuda())
    want = []
    for k in range(4):
        b.step(1)
        want.append(b.reduce())
    assert series.tolist() == want  # the step is bitwise deterministic
    assert dev.cpu().tolist() == want[-1]
    assert a.reduce() == want[-1]


def test_fused_sums_match_standalone_reduction():
    shape = (9, 20, 45)
    M0, solid = synth.channel(shape, 1e-3, seed=4)
    M0 = M0 + 0.0
    M0[1] = 0.01
    s = Solver(shape, lattice=27, tau=0.8, storage="f64", force=(1e-5, 0, 0), mask=solid)
    s.set_moments(M0.cuda())
    s.step(3)
    fused = s.reduce()
    want = dg.reductions(s.moments().cpu(), solid)
    fluid = (~solid).sum().item()
    for k in range(4):
        assert abs(fused[k] - want[k].item()) < 1e-12 * max(1.0, abs(want[k].item()))
    assert abs(fused[5] / 2 / fluid - want[5].item()) < 1e-12


def test_host_buffers_round_trip_and_match_device_path():
    shape = (6, 10, 35)
    M0 = synth.random_moments(shape, seed=30)
    a = Solver(shape, lattice=19, tau=0.7, storage="f32")
    a.set_moments(M0.to(torch.float32).cuda())
    a.step(2)
    b = Solver(shape, lattice=19, tau=0.7, storage="f32")
    b.set_moments(M0.to(torch.float32).pin_memory())
    b.step(2)
    host = b.moments(dtype=torch.float32, device="cpu")
    assert torch.equal(a.moments(dtype=torch.float32).cpu(), host)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("walls", [False, True])
def test_host_transfer_paths_agree(storage, walls):
    """Every way a public state crosses the host link gives the device path's result: pinned host
    memory read and written in place by the encode / decode passes, pageable host memory through the
    idle state buffer (one copy) or, for 16-bit storage, through the staging area in chunks. With
    walls, reading a state back must leave the solid sites of the idle buffer intact."""
    shape = (7, 12, 40)
    M0 = synth.random_moments(shape, seed=31)
    mask = synth.channel_walls(shape) if walls else None
    dt = torch.float64 if storage == "f64" else torch.float32
    ref = Solver(shape, lattice=19, tau=0.7, storage=storage, force=(1e-5, 0.0, 0.0), mask=mask)
    ref.set_moments(M0.to(dt).cuda())
    ref.step(2)
    want = ref.moments(dtype=dt).cpu()
    for pinned_in in (True, False):
        for pinned_out in (True, False):
            s = Solver(shape, lattice=19, tau=0.7, storage=storage, force=(1e-5, 0.0, 0.0), mask=mask)
            src = M0.to(dt)
            s.set_moments(src.pin_memory() if pinned_in else src)
            s.step(1)
            mid = torch.empty((10,) + shape, dtype=dt).pin_memory() if pinned_out else torch.empty((10,) + shape, dtype=dt)
            s.moments(dtype=dt, out=mid)  # read-back between steps must not disturb the next step
            s.step(1)
            out = torch.empty((10,) + shape, dtype=dt).pin_memory() if pinned_out else torch.empty((10,) + shape, dtype=dt)
            got = s.moments(dtype=dt, out=out)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (pinned_in, pinned_out)


def test_instability_is_reported():
    shape = (4, 4, 32)
    M0 = synth.random_moments(shape, seed=2)
    M0[1] += 0.6  # |u| above the 0.4 guard
    s = Solver(shape, lattice=19, tau=0.7, storage="f32")
    s.set_moments(M0.cuda())
    s.step(1)
    with pytest.raises(LBFError) as e:
        s.reduce()
    assert "UNSTABLE" in str(e.value)


def test_bitwise_deterministic():
    shape = (10, 17, 40)
    M0 = synth.random_moments(shape, seed=33)
    outs = []
    sums = []
    for _ in range(2):
        s = Solver(shape, lattice=27, tau=0.6, storage="f32", force=(1e-5, 2e-5, 0))
        s.set_moments(M0.cuda())
        s.step(7)
        outs.append(s.moments(dtype=torch.float32))
        sums.append(s.reduce())
    assert torch.equal(outs[0], outs[1])
    assert sums[0] == sums[1]


def test_step_state_equals_step():
    shape = (8, 9, 33)
    M0 = synth.random_moments(shape, seed=34)
    s = Solver(shape, lattice=19, tau=0.7, storage="f32")
    s.set_moments(M0.cuda())
    a, b = s.new_state(), s.new_state()
    s.copy_state(a)
    s.step_state(a, b)
    s.step(1)
    c = s.new_state()
    s.copy_state(c)
    assert torch.equal(b, c)


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("walls", [False, True])
def test_tma_and_direct_loads_agree(lattice, storage, walls, monkeypatch):
    """The TMA-staged and the directly loaded kernels read the same values and run the same
    arithmetic, compiled separately: the compiler may group multiply-adds differently in the two
    variants (each is deterministic run to run), so one step from the same state must agree to the
    rounding of the storage type - a few units in the last place of FP32/FP64, one or two of
    FP16/BF16 (two where a value near zero comes out of a cancellation: its FP32 rounding error is
    then about one unit of the 16-bit value)."""
    shape = (9, 19, 64)
    M0 = synth.random_moments(shape, seed=40)
    mask = synth.channel_walls(shape) | synth.random_mask(shape, 0.05, seed=41) if walls else None
    outs = []
    for no_tma in (False, True):
        if no_tma:
            monkeypatch.setenv("LBF_NO_TMA", "1")
        s = Solver(shape, lattice=lattice, tau=0.6, storage=storage, force=(1e-5, 0.0, 2e-5), mask=mask)
        s.set_moments(M0.cuda())
        s.step(1)
        st = s.new_state()
        s.copy_state(st)
        outs.append((st.cpu(), s.moments().cpu(), s.reduce()))
    if storage in ("f32", "f64"):
        err = group_errors(outs[0][1], outs[1][1])
        assert max(err.values()) < (1e-6 if storage == "f32" else 1e-14), err
    else:
        # adjacent 16-bit values of one sign differ by one in their bit patterns
        ia = outs[0][0].view(torch.int16).int()
        ib = outs[1][0].view(torch.int16).int()
        assert int((ia - ib).abs().max()) <= 2
        assert (ia != ib).float().mean().item() < 1e-3
    for x, y in zip(outs[0][2], outs[1][2]):
        assert abs(x - y) <= 1e-3 * max(abs(y), 1e-12)
