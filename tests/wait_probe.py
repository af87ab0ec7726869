"""Runs the bounded-wait give-up probe of the LBF_DEBUG library (LBF_LIBRARY) on a small context:
the wait must give up, lbf_synchronize must report LBF_EINTERNAL within milliseconds, and the
context must step normally afterwards. Prints one line; exits non-zero on failure."""
import sys
import time

import torch

import synth
from paper_2609_09160_gb300 import LBFError, Solver, _lbf


def main():
    shape = (4, 10, 32)
    s = Solver(shape, lattice=19, tau=0.8, storage="f32")
    s.set_moments(synth.random_moments(shape, seed=3).cuda())
    s.step(2)
    s.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lbf.lbf_debug_wait_probe(s.ctx, 1000)
    try:
        s.synchronize()
        print("FAIL: the wait did not give up")
        return 1
    except LBFError as e:
        dt = time.perf_counter() - t0
        if e.status != _lbf.LBF_EINTERNAL or "did not complete in time" not in str(e):
            print(f"FAIL: wrong status {e}")
            return 1
    s.step(2)
    s.synchronize()  # reported once: the context is usable again
    out = s.moments()
    if not bool(torch.isfinite(out).all()):
        print("FAIL: non-finite state after the probe")
        return 1
    print(f"ok gave_up_after_s={dt:.6f}")
    return 0 if dt < 1.0 else 1


if __name__ == "__main__":
    sys.exit(main())
