"""Memory floor of the fused step's access pattern on the current GPU.

Builds (in-tree, sm_103a) and runs csrc/stream_floor.cu: the stream-collide kernel's TMA loads and
per-site stores with no arithmetic, for the 30-column output tile the fused kernel uses and for a
128-byte-aligned 32-column tile. One JSON line per variant. Usage:
    python -m paper_2609_09160_gb300.stream_floor [n] [z planes per CTA]
"""
import os
import subprocess
import sys

from . import build as _build

SRC = os.path.join(_build.CSRC, "stream_floor.cu")
EXE = os.path.join(_build.BUILD, "stream_floor")


def compile_floor():
    os.makedirs(_build.BUILD, exist_ok=True)
    if os.path.exists(EXE) and os.path.getmtime(EXE) >= os.path.getmtime(SRC):
        return EXE
    cmd = [_build.nvcc()] + _build.ARCH + ["-O3", "-std=c++17", "-o", EXE, SRC]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on stream_floor.cu:\n{res.stderr[-4000:]}")
    return EXE


def main(argv):
    exe = compile_floor()
    return subprocess.run([exe] + list(argv)).returncode


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
