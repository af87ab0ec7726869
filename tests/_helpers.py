"""Shared test helpers: norm-wise relative errors per field group and GPU solver set-up."""
import torch

# field groups of the public state: p*, u (3), A (6)
GROUPS = {"p": slice(0, 1), "u": slice(1, 4), "A": slice(4, 10)}

# parity tolerances (norm-wise relative, per group) of the GPU path against the FP64 oracle
TOL = {"f64": 1e-12, "f32": 1e-5}


def group_errors(got, want):
    """max |got - want| / max |want| for each field group."""
    got = got.detach().to("cpu", torch.float64)
    want = want.detach().to("cpu", torch.float64)
    out = {}
    for name, sl in GROUPS.items():
        ref = want[sl].abs().max().item()
        out[name] = (got[sl] - want[sl]).abs().max().item() / max(ref, 1e-300)
    return out


def rel_max(got, want):
    got = got.detach().to("cpu", torch.float64)
    want = want.detach().to("cpu", torch.float64)
    return (got - want).abs().max().item() / max(want.abs().max().item(), 1e-300)


def as_f32_exact(M):
    """The FP64 values an FP32 device state holds after upload (storage rounding)."""
    return M.to(torch.float32).to(torch.float64)
