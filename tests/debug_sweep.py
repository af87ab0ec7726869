"""Runs every forward-kernel variant on odd lattice shapes through the library named by
LBF_LIBRARY (the index-checked LBF_DEBUG build in tests/test_gpu_index_checks.py) and prints one
line per case with the status of lbf_synchronize; exits non-zero if any case fails."""
import os
import sys

import torch

import synth
from paper_2609_09160_gb300 import LBFError, Solver

SHAPES = [(1, 1, 1), (3, 5, 7), (5, 9, 31), (4, 17, 36), (6, 10, 64), (9, 26, 40), (3, 8, 33)]
SPLIT_SHAPES = [(3, 30, 64), (2, 41, 40), (5, 26, 96), (9, 26, 40)]


def cases():
    for lattice in (19, 27):
        for storage in ("f64", "f32", "f16", "bf16"):
            for kind in ("periodic", "walls", "field", "two"):
                if kind == "two" and storage in ("f16", "bf16"):
                    continue
                for shape in SHAPES:
                    yield lattice, storage, kind, shape, "cta"
    # the row split (walls at y = 0 and ny - 1: clean rows on the line-aligned kernel, the rows at
    # the walls on the masked 30-column kernel), on shapes whose clean run is long enough for it
    for lattice, storage in ((19, "f32"), (19, "f16"), (27, "f32")):
        for shape in SPLIT_SHAPES:
            yield lattice, storage, "split", shape, "split"
    # the line-aligned kernel (single component, FP32 and 16-bit storage) on the same shapes
    for lattice in (19, 27):
        for storage in ("f32", "f16", "bf16"):
            for kind in ("periodic", "walls", "field"):
                for shape in SHAPES:
                    yield lattice, storage, kind, shape, "aligned"


def run(lattice, storage, kind, shape, kernel):
    os.environ["LBF_KERNEL"] = kernel
    cdt = torch.float64 if storage == "f64" else torch.float32
    kw = {}
    if kind == "walls":
        kw["mask"] = synth.random_mask(shape, 0.2, seed=5)
        kw["force"] = (1e-5, 0.0, 0.0)
    elif kind == "split":
        kw["mask"] = synth.channel_walls(shape)
        kw["force"] = (1e-5, 0.0, 0.0)
    elif kind == "field":
        kw["force_field"] = (1e-5 * torch.randn((3,) + shape, generator=torch.Generator().manual_seed(6))).to(
            device="cuda", dtype=cdt)
    elif kind == "two":
        kw["two_component"] = dict(rho_l=1.0, rho_h=1.0, tau_l=0.9, tau_h=1.1, sigma=0.01, width=3.0, diffusivity=0.1)
    s = Solver(shape, lattice=lattice, tau=0.8, storage=storage, **kw)
    M0 = synth.random_moments(shape, seed=7).to(device="cuda", dtype=cdt)
    if kind == "two":
        s.set_moments(M0, synth.random_field(shape, 0.5, seed=8).abs().clamp(0, 1).to(device="cuda", dtype=cdt))
    else:
        s.set_moments(M0)
    s.step(3)
    s.synchronize()
    out = s.moments()
    assert torch.isfinite(out).all()


def main():
    bad = 0
    for case in cases():
        try:
            run(*case)
            status = "ok"
        except (LBFError, AssertionError) as e:
            status = f"FAIL {e}"
            bad += 1
        print(case, status, flush=True)
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
