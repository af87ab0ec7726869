#!/usr/bin/env python
"""Benchmark of the fused moment-represented LB step on GB300 (MLUPS and HBM roofline).

Headline workload: D3Q19, FP32 storage and arithmetic, 256^3 channel with bounce-back walls on
y = 0 and y = 255, periodic in x and z, uniform body force 1e-6 along x, tau = 0.9, p* = rho - 1
uniform in [-1e-3, 1e-3] (seeded). One step = one launch of the fused stream-collide kernel with
the FP64 conservation sums fused in. The two moment buffers (2 x 671 MB) exceed the 129 MB L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick]

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on a bounded sample
of the same workload on the host cores. Under torchrun every rank runs its own replica on its own
GPU (the path is not sharded); the time is the max over ranks and the value the sum of all
replicas' lattice updates per second.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM GB/s (D3Q19/27, FP32 vs FP16-stored); adjoint/forward time ratio"
WORKLOAD = ("D3Q19 regularized, moment-represented, FP32, 256^3 channel: bounce-back walls y=0,255, periodic x/z, "
            "body force 1e-6 along x, tau=0.9, p* = rho-1 ~ U[-1e-3,1e-3] seed 1")
SHAPE = (256, 256, 256)
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}


def algorithmic_bytes(storage, mask=False, field=False):
    """Per lattice update: each of the 10 stored fields read once and written once, plus the
    mask byte and a per-site FP32 force field when present."""
    b = 20 * STORAGE_BYTES[storage]
    if mask:
        b += 1
    if field:
        b += 3 * (8 if storage == "f64" else 4)
    return b


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha1()
    for name in ("lattice.cuh", "stream_collide.cuh", "stream_collide_aligned.cuh", "tma.cuh"):
        with open(os.path.join(ROOT, "paper_2609_09160_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(workload_key):
    """dram bytes of one step (all its launches) recorded from an ncu capture of the current kernel
    source, else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha()
    for line in open(path):
        parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if parts.get("workload") == workload_key and parts.get("kernel_sha") == sha:
            return float(parts.get("bytes_per_step", parts.get("bytes_per_launch")))
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu_id)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3].split()[0]) for r in rows if r[3].split() and r[3].split()[0].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w": statistics.median(pw) if pw else None}


def gpu_identifier(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(dev)


LATTICE_NAME = {19: "D3Q19", 27: "D3Q27", 127: "D3Q27h"}
# FP32 bytes per site of a two-component step beyond the 80 B of the moments, over its three
# kernels: the fused step reads phi and F at t and t+1 (4 + 12 + 4 + 12), the phase-field advance
# reads phi, u, G and writes phi (4 + 12 + 12 + 4), the forces read phi and write F and G (4 + 24)
TWO_COMPONENT_EXTRA_BYTES = 32 + 32 + 28
# with a density contrast the forces kernel also writes grad phi (12), the fused step reads it (12)
# and writes the total force of the new state back (12); walls add the mask byte to the advance
CONTRAST_EXTRA_BYTES = 36 + 1

WORKLOADS = {
    # key: (lattice, storage, builder) -- the headline is "channel256"
    "channel256": (19, "f32", "channel"),
    "tg512_d3q27_f32": (27, "f32", "tg512"),
    "tg512_d3q27_f16": (27, "f16", "tg512"),
    "tg512_d3q27_bf16": (27, "bf16", "tg512"),
    "tg512_d3q19_f32": (19, "f32", "tg512"),
    "tg512_d3q19_f16": (19, "f16", "tg512"),
    "tg512_d3q27h_f32": (127, "f32", "tg512"),
    "tg512_d3q27h_f16": (127, "f16", "tg512"),
    # 256^3 periodic Taylor-Green: the same kernels on a lattice small enough for ncu captures
    "tg256_d3q19_f32": (19, "f32", "tg256"),
    "tg256_d3q27_f32": (27, "f32", "tg256"),
    "tg256_d3q27h_f32": (127, "f32", "tg256"),
    "tg256_d3q19_f16": (19, "f16", "tg256"),
    "tg256_d3q27_f16": (27, "f16", "tg256"),
    "droplet128": (19, "f32", "droplet"),
    "layered512": (19, "f32", "layered"),
    "adjoint128": (19, "f32", "adjoint"),
}


def workload_solver(torch, device, key):
    """Solver + initial state of a named workload (returns solver, public state, mask)."""
    lattice, storage, kind = WORKLOADS[key]
    if kind == "channel":
        return channel_solver(torch, device, storage, lattice)
    if kind == "droplet":
        return droplet_solver(torch, device)
    if kind == "layered":
        s, M0, phi0 = layered_solver(torch, device)
        s._phi0 = phi0
        return s, M0, None
    import synth
    from paper_2609_09160_gb300 import Solver

    n = 512 if kind == "tg512" else 256
    M0 = synth.taylor_green_perturbed(n, 0.04, 0.55, 0.01, seed=3, dtype=torch.float32, device=device)
    s = Solver((n, n, n), lattice=lattice, tau=0.55, storage=storage, device=device)
    return s, M0, None


def droplet_solver(torch, device, n=128):
    """Two-component static droplet: R = 20, W = 4, sigma = 0.03, D = 0.1, equal densities, tau = 1."""
    import synth
    from paper_2609_09160_gb300 import Solver

    shape = (n, n, n)
    s = Solver(shape, lattice=19, storage="f32", device=device,
               two_component=dict(rho_l=1.0, rho_h=1.0, tau_l=1.0, tau_h=1.0, sigma=0.03, width=4.0, diffusivity=0.1))
    phi0 = synth.droplet(shape, 20.0, 4.0, dtype=torch.float32, device=device)
    M0 = torch.zeros((10,) + shape, dtype=torch.float32, device=device)
    s._phi0 = phi0
    return s, M0, None


def layered_solver(torch, device, nx=512, ny=1024, nz=8):
    """Layered two-phase Poiseuille flow (Sec. 4, 512 x 8 x 1024): walls at x = 0 and nx - 1, light
    phase (rho 0.5, nu 0.05) for x < nx/2, heavy phase (rho 1.5, nu 0.4) above, tanh interface of
    width 4, body acceleration 1e-7 along the layers, fluid at rest. The paper's flow direction
    (1024 sites) is laid along y and its thin periodic direction (8 sites) along z, where the
    kernels march in planes, so that no tile of 7 or 8 rows is left mostly empty."""
    from paper_2609_09160_gb300 import Solver

    shape = (nz, ny, nx)
    x = torch.arange(nx, dtype=torch.float32, device=device)
    phi0 = (0.5 * (1 + torch.tanh(2 * (x - nx / 2) / 4.0))).reshape(1, 1, nx).expand(shape).contiguous()
    mask = torch.zeros(shape, dtype=torch.bool)
    mask[..., 0] = mask[..., -1] = True
    tc = dict(rho_l=0.5, rho_h=1.5, tau_l=3 * 0.05 + 0.5, tau_h=3 * 0.4 + 0.5, sigma=0.03, width=4.0,
              diffusivity=0.1, body_accel=(0.0, 1e-7, 0.0))
    s = Solver(shape, lattice=19, storage="f32", two_component=tc, mask=mask, device=device)
    M0 = torch.zeros((10,) + shape, dtype=torch.float32, device=device)
    return s, M0, phi0


def adjoint_rollout(torch, device, T=500, K=50, reps=2):
    """Config-5 rollout: 128(x) x 64(y) x 64(z) channel, per-site force N(0, 1e-12) on the fluid,
    loss = mean |u(T) - u_target|^2, checkpoints every K steps. Returns (forward s, backward s)."""
    import synth
    from paper_2609_09160_gb300 import Solver, rollout

    shape = (64, 64, 128)
    mask = synth.channel_walls(shape)
    F = synth.random_field(shape, 1e-6, seed=70, mask=mask).to(device=device, dtype=torch.float32)
    F.requires_grad_(True)
    u_tgt = synth.random_field(shape, 1e-4, seed=71).to(device=device, dtype=torch.float32)
    fluid = (~mask).to(device=device, dtype=torch.float32)
    s = Solver(shape, lattice=19, tau=0.9, storage="f32", force_field=F.detach(), mask=mask, device=device)
    M0 = torch.zeros((10,) + shape, dtype=torch.float32, device=device)
    times = []
    for _ in range(reps):  # the first repetition warms up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        MT = rollout(F, M0, s, T, K)
        d = (MT[1:4] - u_tgt) * fluid
        L = (d * d).sum() / fluid.sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        F.grad = None
        times.append((t1 - t0, t2 - t1))
    return times[-1], s.N


def channel_solver(torch, device, storage="f32", lattice=19, shape=SHAPE, populations=False):
    import synth
    from paper_2609_09160_gb300 import Solver

    M0, solid = synth.channel(shape, 1e-3, seed=1, dtype=torch.float32)
    s = Solver(shape, lattice=lattice, tau=0.9, storage=storage, force=(1e-6, 0.0, 0.0), mask=solid, device=device,
               populations=populations)
    return s, M0, solid


def time_steps(torch, s, steps, warmup, barrier=None):
    """Device time of `steps` steps on the solver's stream (Solver.kernels_per_step launches each;
    launches on the library's side stream are joined back to it before the step ends)."""
    for _ in range(warmup):
        s.step(1)
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(s.stream)
    for _ in range(steps):
        s.step(1)
    end.record(s.stream)
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    return start.elapsed_time(end) / 1e3


def e2e_measure(torch, device, steps):
    """Same metric through the public API with host buffers: upload the public state from pinned
    host memory, run the steps copying the FP64 conservation sums of every step to pinned host
    memory (one 48-byte device-to-host copy per step, Solver.reduce_async: no host wait between
    steps), download the final state to pinned host memory; the host checks the last sums after
    the final synchronisation. "blocking_reduce" is the same leg with Solver.reduce (the host waits
    for every step's sums before launching the next step)."""
    s, M0, _ = channel_solver(torch, device)
    host_in = M0.pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    series = torch.empty((steps, 6), dtype=torch.float64).pin_memory()
    s.set_moments(host_in)
    s.step(3)
    s.reduce()
    torch.cuda.synchronize()
    n = M0[0].numel()
    nbytes = host_in.numel() * host_in.element_size()

    def leg(blocking):
        t0 = time.perf_counter()
        s.set_moments(host_in)
        for k in range(steps):
            s.step(1)
            if blocking:
                s.reduce()
            else:
                s.reduce_async(series[k])
        s.moments(out=host_out)
        s.synchronize()
        t = time.perf_counter() - t0
        if not blocking and not all(math.isfinite(v) for v in series[steps - 1].tolist()):
            raise RuntimeError("non-finite sums in the end-to-end leg")
        return n * steps / t / 1e6

    value = leg(False)
    blocking = leg(True)
    return {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": nbytes / steps,
            "d2h_bytes_per_step": 48 + nbytes / steps, "blocking_reduce": round(blocking, 2)}


def _time_oracle_steps(step, target_seconds, max_steps):
    """Run step() until target_seconds have passed (at least 2, at most max_steps calls)."""
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (steps < 2 or time.perf_counter() - t0 < target_seconds):
        step()
        steps += 1
    return steps, time.perf_counter() - t0


def cpu_baseline_oracle(target_seconds=10.0):
    """The FP64 oracle as it stands, timed on the host cores: the headline sample (a 256x256x4
    z-slab of the channel) on all cores and on one core, a 128x128x4 slab of the D3Q27 512^3
    Taylor-Green workload, and the config-5 rollout (forward and its autograd adjoint) on a
    128x64x4 slab of the adjoint channel. Each leg runs for about target_seconds."""
    import torch

    import oracle
    import synth

    all_cores = torch.get_num_threads()

    def channel_leg(threads, seconds, max_steps):
        shape = (4, 256, 256)
        M0, solid = synth.channel(shape, 1e-3, seed=1)
        F = oracle.lbm.as_field((1e-6, 0.0, 0.0), shape)
        rho = oracle.lbm.as_scalar_field(1.0, shape)
        om = oracle.lbm.as_scalar_field(oracle.lbm.omega_from_tau(0.9), shape)
        st = {"f": oracle.lbm.populations_from_moments(oracle.D3Q19, M0, F, rho)}
        torch.set_num_threads(threads)
        try:
            steps, t = _time_oracle_steps(lambda: st.update(f=oracle.lbm.step(oracle.D3Q19, st["f"], F, rho, om, solid)),
                                          seconds, max_steps)
        finally:
            torch.set_num_threads(all_cores)
        return {"value": round(256 * 256 * 4 * steps / t / 1e6, 4), "unit": "MLUPS", "cores": threads,
                "sample": f"{steps} population-form FP64 D3Q19 steps on a 256x256x4 (x,y,z) slab of the channel"}

    def d3q27_leg(seconds):
        shape = (4, 128, 128)
        M = synth.taylor_green_perturbed(128, 0.04, 0.55, 0.01, seed=3)[:, :4].contiguous()
        F = oracle.lbm.as_field((0.0, 0.0, 0.0), shape)
        rho = oracle.lbm.as_scalar_field(1.0, shape)
        om = oracle.lbm.as_scalar_field(oracle.lbm.omega_from_tau(0.55), shape)
        st = {"f": oracle.lbm.populations_from_moments(oracle.D3Q27, M, F, rho)}
        steps, t = _time_oracle_steps(lambda: st.update(f=oracle.lbm.step(oracle.D3Q27, st["f"], F, rho, om, None)),
                                      seconds, 200)
        return {"value": round(128 * 128 * 4 * steps / t / 1e6, 4), "unit": "MLUPS", "cores": all_cores,
                "sample": f"{steps} population-form FP64 D3Q27 steps on a 128x128x4 slab of the 128^3 "
                          "Taylor-Green + perturbation workload"}

    def adjoint_leg(steps=8):
        shape = (4, 64, 128)
        mask = synth.channel_walls(shape)
        F = synth.random_field(shape, 1e-6, seed=70, mask=mask)
        u_tgt = synth.random_field(shape, 1e-4, seed=71)
        M0 = torch.zeros((10,) + shape, dtype=torch.float64)
        t0 = time.perf_counter()
        oracle.adjoint.rollout_loss(oracle.D3Q19, M0, F, steps, 0.9, u_tgt, mask)
        t1 = time.perf_counter()
        oracle.adjoint.rollout_gradient(oracle.D3Q19, M0, F, steps, 0.9, u_tgt, mask)
        t2 = time.perf_counter()
        fwd, both = t1 - t0, t2 - t1
        n = 128 * 64 * 4
        return {"forward_MLUPS": round(n * steps / fwd / 1e6, 4), "adjoint_over_forward": round((both - fwd) / fwd, 3),
                "cores": all_cores,
                "sample": f"config-5 rollout of {steps} steps on a 128x64x4 (x,y,z) slab of the adjoint channel: "
                          "oracle forward, then forward + autograd backward"}

    head = channel_leg(all_cores, target_seconds, 50)
    legs = {"channel256_slab_1core": channel_leg(1, target_seconds / 2, 10),
            "tg128_d3q27_slab": d3q27_leg(target_seconds / 2),
            "adjoint_config5_slab": adjoint_leg()}
    return {"value": head["value"], "unit": "MLUPS", "cores": all_cores, "kind": "oracle", "sample": head["sample"],
            "cores_listed": [all_cores, 1], "legs": legs}


def extras(torch, device, quick):
    """Secondary rows: D3Q27, D3Q19 and D3Q27h 512^3 in every storage dtype, the population-form
    channel, two-component, FP64, adjoint ratio."""
    import synth
    from paper_2609_09160_gb300 import Solver, rollout

    out = {}
    peak, _ = measured_peaks()

    def rate(s, steps, warmup, bytes_per_lup):
        t = time_steps(torch, s, steps, warmup)
        n = s.N
        mlups = n * steps / t / 1e6
        return {"MLUPS": round(mlups, 1), "algorithmic_GBps": round(bytes_per_lup * mlups / 1e3, 1),
                "hbm_frac_of_measured": round(bytes_per_lup * mlups / 1e3 / peak, 3), "steps": steps}

    n = 512
    M0 = synth.taylor_green_perturbed(n, 0.04, 0.55, 0.01, seed=3, dtype=torch.float32, device=device)
    for lattice in (27, 19, 127):  # 127: D3Q27h (complete Hermite basis)
        for storage in ("f32", "f16", "bf16"):
            s = Solver((n, n, n), lattice=lattice, tau=0.55, storage=storage, device=device)
            s.set_moments(M0)
            out[f"tg512_{LATTICE_NAME[lattice].lower()}_{storage}"] = rate(s, 30 if quick else 100, 5,
                                                                           algorithmic_bytes(storage))
            del s
            torch.cuda.empty_cache()
    del M0
    torch.cuda.empty_cache()

    # the same channel in the population representation (Q = 19 FP32 fields per buffer, 152 B + mask
    # per update): the layout the paper's moment representation replaces
    s, M0, _ = channel_solver(torch, device, populations=True)
    s.set_moments(M0.to(device))
    r = rate(s, 50 if quick else 200, 5, 2 * 19 * 4 + 1)
    r["note"] = "population-form reference kernel (lbf_params.populations), same scheme and workload as the headline"
    out["channel256_d3q19_f32_populations"] = r
    del s, M0
    torch.cuda.empty_cache()

    # two-component droplet, 128^3, R = 20, equal densities, tau = 1 (config of the Laplace test)
    s, M0, _ = droplet_solver(torch, device)
    s.set_moments(M0, s._phi0)
    r = rate(s, 50 if quick else 200, 5, TWO_COMPONENT_EXTRA_BYTES + algorithmic_bytes("f32"))
    r["note"] = "3 kernels per step (phase field advance, forces, fused LB)"
    out["droplet128_d3q19_f32"] = r
    del s, M0
    torch.cuda.empty_cache()

    # density and viscosity contrast: the layered two-phase Poiseuille flow of Sec. 4 at the paper's
    # size, 512 (x, walls at x = 0 and 511) x 1024 (y, flow direction) x 8 (z), rho 0.5 / 1.5,
    # nu 0.05 / 0.4, W = 4, sigma = 0.03, body acceleration 1e-7 along the layers, interface at x = 256
    s, M0, phi0 = layered_solver(torch, device)
    s.set_moments(M0, phi0)
    r = rate(s, 50 if quick else 200, 5,
             TWO_COMPONENT_EXTRA_BYTES + CONTRAST_EXTRA_BYTES + algorithmic_bytes("f32", mask=True))
    r["note"] = "3 kernels per step; pressure and viscous-gradient forces in the fused step"
    out["layered512x1024x8_d3q19_f32_contrast"] = r
    del s, M0, phi0

    # FP64 parity mode: 32^3 Taylor-Green (launch-latency bound at this size)
    s = Solver((32, 32, 32), lattice=19, tau=0.8, storage="f64", device=device)
    s.set_moments(synth.taylor_green(32, 0.02, 0.8, device=device))
    out["tg32_d3q19_f64"] = rate(s, 100, 5, algorithmic_bytes("f64"))
    del s

    # adjoint / forward time ratio: 128x64x64 channel, per-site force, 500 steps, checkpoints every 50
    T = 100 if quick else 500
    (tf, tb), n = adjoint_rollout(torch, device, T=T)
    out["adjoint_128x64x64_d3q19_f32"] = {"forward_s": round(tf, 4), "backward_s": round(tb, 4),
                                          "ratio": round(tb / tf, 3), "steps": T, "checkpoint_every": 50,
                                          "forward_MLUPS": round(n * T / tf / 1e6, 1)}
    return out


class NvmlEnergy:
    """Board energy counter of one GPU through NVML (nvmlDeviceGetTotalEnergyConsumption, mJ since
    the driver loaded): the quantity the paper integrates for its energy per lattice update. A
    read-only query; None where NVML is not available."""

    def __init__(self, uuid):
        import ctypes

        self.lib = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(uuid.encode()), ctypes.byref(h)) != 0:
                return
            self.lib, self.handle, self.ct = lib, h, ctypes
        except Exception:
            self.lib = None

    def read_mj(self):
        if self.lib is None:
            return None
        v = self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.handle, self.ct.byref(v)) != 0:
            return None
        return int(v.value)


def energy_leg(torch, s, gpu_id, seconds_per_step, target_seconds=2.5):
    """Energy per lattice update (the paper's metric, Sec. 5): the NVML energy counter read before
    and after at least ~2.5 s of steps, divided by the lattice updates; board power sampled by
    nvidia-smi over the same steps. Returns None without NVML."""
    meter = NvmlEnergy(gpu_id)
    if meter.lib is None:
        return {"nJ_per_lup": None, "source": "NVML not available"}
    steps = max(200, int(target_seconds / max(seconds_per_step, 1e-6)))
    s.step(10)
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        e0 = meter.read_mj()
        t0 = time.perf_counter()
        s.step(steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e1 = meter.read_mj()
    clocks = clk.summary()
    if e0 is None or e1 is None or e1 <= e0:
        return {"nJ_per_lup": None, "source": "NVML energy counter did not advance"}
    joules = (e1 - e0) / 1e3
    return {"nJ_per_lup": round(joules / (s.N * steps) * 1e9, 4), "power_w": round(joules / (t1 - t0), 1),
            "seconds": round(t1 - t0, 3), "steps": steps, "clocks_during": clocks,
            "source": "NVML nvmlDeviceGetTotalEnergyConsumption, difference over the steps of this leg"}


def max_over_ranks(torch, dist, t, device):
    """The job's time: the slowest rank's (every rank gets it)."""
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return tt.item()


def replicas_mlups(world, sites_per_rank, steps, t):
    """Whole-job throughput of `world` independent replicas of `sites_per_rank` sites, `steps`
    steps each, finished after `t` seconds (weak scaling: the work per rank is fixed)."""
    return world * sites_per_rank * steps / t / 1e6


def kernel_label(s, lattice, storage, kind):
    """The kernels one timed step runs (the roofline unit is one step: its launches together)."""
    lat = LATTICE_NAME[lattice]
    walls = kind in ("channel", "layered")
    if s.kernels_per_step == 2 and kind == "channel":
        return (f"k_stream_collide_al<{lat},{storage},periodic> on the rows clear of the walls + "
                f"k_stream_collide<{lat},{storage},mask> on the rows near them")
    fused = (f"k_stream_collide<{lat},{storage},{'mask' if walls else 'periodic'}>" if walls or kind == "droplet"
             else f"k_stream_collide_al or k_stream_collide<{lat},{storage},periodic> (the library's choice)")
    if kind in ("droplet", "layered"):
        return f"k_phase_advance + k_phase_forces + {fused}"
    return fused


def run_ours(args):
    import torch

    from paper_2609_09160_gb300 import build as _build

    _build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    barrier = None
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        barrier = dist.barrier
    if WORKLOADS[args.workload][2] == "adjoint":
        (tf, tb), n = adjoint_rollout(torch, device)
        if rank == 0:
            print(json.dumps({"metric": "adjoint/forward time ratio", "value": round(tb / tf, 3), "unit": "ratio",
                              "forward_s": tf, "backward_s": tb, "forward_MLUPS": n * 500 / tf / 1e6,
                              "higher_is_better": False, "workload": args.workload}), flush=True)
        return
    s, M0, solid = workload_solver(torch, device, args.workload)
    if WORKLOADS[args.workload][2] in ("droplet", "layered"):
        s.set_moments(M0, s._phi0)
    else:
        s.set_moments(M0.to(device))
    del M0
    with ClockSampler(gpu_identifier(torch, device)) as clk:
        t = time_steps(torch, s, args.steps, args.warmup, barrier)
    clocks = clk.summary()
    if world > 1:
        t = max_over_ranks(torch, dist, t, device)
    n = s.N
    value = replicas_mlups(world, n, args.steps, t)
    sums = s.reduce()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    lattice, storage, kind = WORKLOADS[args.workload]
    bpl = algorithmic_bytes(storage, mask=(kind == "channel"))
    if kind == "droplet":
        bpl += TWO_COMPONENT_EXTRA_BYTES
    if kind == "layered":
        bpl = algorithmic_bytes(storage, mask=True) + TWO_COMPONENT_EXTRA_BYTES + CONTRAST_EXTRA_BYTES
    t_launch = t / args.steps
    achieved = bpl * n / t_launch / 1e9
    traffic = ncu_traffic(args.workload)
    desc = {"channel": WORKLOAD,
            "droplet": "two-component D3Q19 FP32 128^3 static droplet R=20, W=4, sigma=0.03, D=0.1, tau=1",
            "layered": ("two-component D3Q19 FP32 layered flow with density contrast 512(x) x 1024(y) x 8(z): walls "
                        "x=0,511, rho 0.5/1.5, nu 0.05/0.4, W=4, body acceleration 1e-7 along y"),
            "tg512": (f"{LATTICE_NAME[lattice]} {storage.upper()} storage, 512^3 periodic Taylor-Green U0=0.04 + random-phase "
                      "perturbation RMS 0.01 (seed 3), tau=0.55"),
            "tg256": (f"{LATTICE_NAME[lattice]} {storage.upper()} storage, 256^3 periodic Taylor-Green U0=0.04 + random-phase "
                      "perturbation RMS 0.01 (seed 3), tau=0.55")}[kind]
    shape_xyz = {"channel": [256, 256, 256], "droplet": [128, 128, 128], "tg512": [512, 512, 512], "tg256": [256, 256, 256],
                 "layered": [512, 1024, 8]}[kind]
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t * 1e3 / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if storage == "f64" else "f32", "data": "synthetic",
        "config": {"workload": desc, "lattice": LATTICE_NAME[lattice], "shape_xyz": shape_xyz, "storage": storage,
                   "l2": "inputs larger than L2 (two moment buffers of >= 671 MB), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": kernel_label(s, lattice, storage, kind),
                     "bytes_per_lup": bpl, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"},
        "gpu_launches": args.steps * s.kernels_per_step,
        "clocks": clocks,
        "sums_after": {"sum_p": sums[0], "sum_ux": sums[1]},
    }
    if world == 1 and not args.kernel_only:
        # energy per lattice update: NVML energy counter over a separate leg of >= 2.5 s of steps
        # (the timed region above can be far shorter than the power sampling interval)
        line["energy"] = energy_leg(torch, s, gpu_identifier(torch, device), t / args.steps)
    if world == 1 and not args.kernel_only and args.workload == "channel256":
        line["e2e"] = e2e_measure(torch, device, args.steps)
        line["cpu_baseline"] = cpu_baseline_oracle()
        if not args.quick:
            try:
                line["extra"] = extras(torch, device, args.quick)
            except Exception as exc:  # keep the headline line even if a secondary row fails
                line["extra"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle as it stands, on the host cores: each step is one oracle step on a
    one-plane (256 x 256 x 1, periodic in z) sample of the channel workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    import oracle
    import synth

    shape = (1, 256, 256)
    M0, solid = synth.channel(shape, 1e-3, seed=1)
    lat = oracle.D3Q19
    F = oracle.lbm.as_field((1e-6, 0.0, 0.0), shape)
    rho = oracle.lbm.as_scalar_field(1.0, shape)
    om = oracle.lbm.as_scalar_field(oracle.lbm.omega_from_tau(0.9), shape)
    f = oracle.lbm.populations_from_moments(lat, M0, F, rho)
    for _ in range(args.warmup):
        f = oracle.lbm.step(lat, f, F, rho, om, solid)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.lbm.step(lat, f, F, rho, om, solid)
    t = time.perf_counter() - t0
    n = shape[0] * shape[1] * shape[2]
    value = n * args.steps / t / 1e6
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "D3Q19", "shape_xyz": [256, 256, 256], "storage": "f64",
                   "sample": "one 256x256 plane per step (periodic in z)"},
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} FP64 population-form steps on a 256x256x1 slab of the channel"},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the secondary rows")
    ap.add_argument("--kernel-only", action="store_true",
                    help="only the device-timed steps (no e2e, CPU baseline or secondary rows): for profiling")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="channel256")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
