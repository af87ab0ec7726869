"""The population-form reference representation (lbf_params.populations): the context stores the
Q post-collision populations of Eq. (pullLB) instead of the 10 moments and steps them with the
same regularized collision. Its results must match the FP64 oracle like the moment path does, and
match the moment representation itself; the moment and population forms are the same scheme
(the 4^3 brute-force pin of the oracle, Sec. 2)."""
import pytest
import torch

from paper_2609_09160_gb300 import LBFError, Solver, _lbf

from _helpers import TOL, group_errors
from test_gpu_step import CDT, make_case, run_oracle

pytestmark = pytest.mark.gpu


def run(lattice, storage, shape, M0, force, field, mask, steps, tau, populations):
    ff = None if field is None else field.to(device="cuda", dtype=CDT[storage]).contiguous()
    s = Solver(shape, lattice=lattice, tau=tau, storage=storage, force=force, force_field=ff, mask=mask,
               populations=populations)
    s.set_moments(M0.cuda())
    s.step(steps)
    return s.moments(), s


@pytest.mark.parametrize("lattice", [19, 27])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case", ["periodic", "uniform_force", "walls_field"])
def test_population_representation_matches_oracle_and_moment_form(lattice, storage, case):
    shape = (11, 13, 37)
    M0, force, field, mask = make_case(case, shape, storage, seed=lattice + 3)
    got, sp = run(lattice, storage, shape, M0, force, field, mask, 5, 0.7, True)
    want = run_oracle(lattice, storage, M0, force, field, mask, 5, 0.7)
    err = group_errors(got, want)
    assert max(err.values()) < TOL[storage], err
    mom, sm = run(lattice, storage, shape, M0, force, field, mask, 5, 0.7, False)
    err = group_errors(got, mom)
    assert max(err.values()) < TOL[storage], err
    # conservation sums of the fused reduction agree between the representations
    rp, rm = sp.reduce(), sm.reduce()
    scale = [abs(M0[0]).sum().item(), *(abs(M0[1 + a]).sum().item() for a in range(3))]
    tol = 1e-12 if storage == "f64" else 1e-6
    for k in range(4):
        assert abs(rp[k] - rm[k]) <= tol * scale[k], (k, rp[k], rm[k])


def test_population_state_holds_q_fields_and_steps_in_place():
    shape = (6, 7, 33)
    M0, force, field, mask = make_case("walls_field", shape, "f32", seed=5)
    for lattice in (19, 27):
        _, s = run(lattice, "f32", shape, M0, force, field, mask, 0, 0.8, True)
        assert s.state_bytes == lattice * 6 * 7 * 33 * 4
        a, b = s.new_state(), s.new_state()
        s.copy_state(a)
        b.copy_(a)
        s.step_state(a, b)  # one step between caller buffers
        s.step(1)
        c = s.new_state()
        s.copy_state(c)
        assert torch.equal(b, c)


def test_population_representation_refuses_what_it_does_not_build():
    shape = (4, 4, 8)
    with pytest.raises(LBFError) as e:
        Solver(shape, lattice=19, storage="f16", populations=True)
    assert e.value.status == _lbf.LBF_ENOTSUP
    s = Solver(shape, lattice=19, storage="f32", populations=True)
    s.set_moments(torch.zeros((10,) + shape, dtype=torch.float32, device="cuda"))
    lam = torch.zeros((10,) + shape, dtype=torch.float32, device="cuda")
    g = torch.zeros((3,) + shape, dtype=torch.float64, device="cuda")
    st = s.new_state()
    s.copy_state(st)
    with pytest.raises(LBFError) as e:
        s.adjoint_step(st, st, lam, lam.clone(), g)
    assert e.value.status == _lbf.LBF_ENOTSUP
