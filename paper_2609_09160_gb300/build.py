"""In-tree build of the CUDA library liblbf.so for sm_103a (GB300).

The translation units are compiled in parallel with nvcc and linked with the static CUDA
runtime, so the library only needs the driver at run time. `python -m
paper_2609_09160_gb300.build` rebuilds when a source or header is newer than the library.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbf.so")
SOURCES = ["api.cu", "static_step.cu", "kernels.cu"]
# kernels.cu is compiled once per (lattice, storage) pair; each object holds that pair's kernels
KERNEL_UNITS = [(q, s) for q in (19, 27, 127) for s in range(4)]  # 127: D3Q27h
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-O2", "-I", os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbf.so")
    return exe


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return files


STAMP = os.path.join(BUILD, "flags.txt")
# index-checked variant (LBF_DEBUG): its own objects and library, never loaded by default
DEBUG_BUILD = os.path.join(PKG, "_build_debug")
DEBUG_LIB = os.path.join(PKG, "liblbf_debug.so")


def up_to_date(tuning=(), lib=LIB, stamp=STAMP):
    if not os.path.exists(lib) or not os.path.exists(stamp):
        return False
    if open(stamp).read() != " ".join(tuning):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _units():
    """(source, object name, defines) of every translation unit."""
    units = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        if s == "kernels.cu":
            for q, st in KERNEL_UNITS:
                units.append((src, f"kernels_q{q}_s{st}", [f"-DLBF_TU_LATTICE={q}", f"-DLBF_TU_STORAGE={st}"]))
        else:
            units.append((src, os.path.splitext(s)[0], []))
    return units


def _compile(unit, extra, build_dir=BUILD):
    src, name, defines = unit
    obj = os.path.join(build_dir, name + ".o")
    log = os.path.join(build_dir, name + ".log")
    cmd = [nvcc()] + NVCC_FLAGS + defines + extra + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + res.stdout + res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {name}:\n{res.stderr[-4000:]}")
    return obj


def build(force=False, verbose_ptxas=False, debug=False):
    """Compile liblbf.so in place; returns its path. LBF_NVCC_EXTRA (space-separated nvcc flags,
    e.g. tile-size defines) is appended for tuning builds and forces a rebuild. debug=True builds
    liblbf_debug.so instead: the same library with every index of the fused step checked
    (LBF_DEBUG), for tests; load it by pointing LBF_LIBRARY at it."""
    tuning = os.environ.get("LBF_NVCC_EXTRA", "").split()
    build_dir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    stamp = os.path.join(build_dir, "flags.txt")
    if not force and up_to_date(tuning, lib, stamp):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + tuning + (["-DLBF_DEBUG"] if debug else [])
    units = _units()
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda u: _compile(u, extra, build_dir), units))
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr[-4000:]}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(" ".join(tuning))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
