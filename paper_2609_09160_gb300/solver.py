"""Solver: a context of the C library with its device workspace held by a torch tensor.

PyTorch only provides memory and the stream; every step of the method runs in liblbf.so.
All calls are ordered on the torch stream that was current when the Solver was created.
"""
import ctypes

import torch

from . import _lbf

STORAGE = {"f64": _lbf.LBF_F64, "f32": _lbf.LBF_F32, "f16": _lbf.LBF_F16, "bf16": _lbf.LBF_BF16}
_TORCH_DTYPE = {_lbf.LBF_F64: torch.float64, _lbf.LBF_F32: torch.float32}


def _dtype_code(dtype):
    if dtype == torch.float64:
        return _lbf.LBF_F64
    if dtype == torch.float32:
        return _lbf.LBF_F32
    raise ValueError("moments are exchanged as float64 or float32")


class Solver:
    """Moment-represented LB solver on one GPU.

    shape = (nz, ny, nx); lattice 19, 27 or '27h' (= 127, D3Q27 with the complete Hermite basis);
    storage 'f64' | 'f32' | 'f16' | 'bf16'.
    force: uniform 3-vector; force_field: CUDA tensor (3, nz, ny, nx) in the compute dtype
    (float64 for 'f64' storage, else float32), kept by reference; mask: bool/uint8 (nz, ny, nx),
    nonzero = solid. two_component: dict(rho_l, rho_h, tau_l, tau_h, sigma, width, diffusivity and
    optionally body_accel, a uniform body acceleration).
    """

    def __init__(self, shape, lattice=19, tau=0.8, storage="f32", force=(0.0, 0.0, 0.0), force_field=None,
                 mask=None, two_component=None, scale_hint=None, rounding="stochastic", populations=False,
                 device=None):
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("the solver runs on a CUDA device only")
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.compute_dtype = torch.float64 if self.storage == _lbf.LBF_F64 else torch.float32
        p = _lbf.lbf_params()
        lattice = _lbf.LBF_D3Q27H if str(lattice).lower() in ("27h", "d3q27h") else int(lattice)
        p.lattice, p.nx, p.ny, p.nz, p.storage = lattice, nx, ny, nz, self.storage
        p.tau = float(tau)
        for a in range(3):
            p.force[a] = float(force[a])
        self._keep = []
        if force_field is not None:
            if force_field.dtype != self.compute_dtype or not force_field.is_cuda or not force_field.is_contiguous():
                raise ValueError("force_field must be a contiguous CUDA tensor in the compute dtype")
            p.force_field = force_field.data_ptr()
            self._keep.append(force_field)
        self.force_field = force_field
        self.mask = None
        if mask is not None:
            m = torch.as_tensor(mask).to(device="cpu", dtype=torch.uint8).contiguous()
            self.mask = m.bool()
            p.mask = m.data_ptr()
            self._mask_host = m
        self.two_component = two_component is not None
        if two_component is not None:
            tc = dict(two_component)
            p.two_component = 1
            p.rho_l, p.rho_h = float(tc.get("rho_l", 1.0)), float(tc.get("rho_h", 1.0))
            p.tau_l, p.tau_h = float(tc["tau_l"]), float(tc["tau_h"])
            p.sigma, p.width, p.diffusivity = float(tc["sigma"]), float(tc["width"]), float(tc["diffusivity"])
            for k, v in enumerate(tc.get("body_accel", (0.0, 0.0, 0.0))):
                p.body_accel[k] = float(v)
        if scale_hint is not None:
            for a in range(3):
                p.scale_hint[a] = float(scale_hint[a])
        p.rounding = {"stochastic": _lbf.LBF_ROUND_STOCHASTIC, "nearest": _lbf.LBF_ROUND_NEAREST}[rounding]
        p.populations = 1 if populations else 0
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            p.stream = self.stream.cuda_stream
            self.params = p
            nbytes = _lbf.lbf_workspace_bytes(p)
            if nbytes == 0:
                _lbf._check(_lbf.lbf_validate(p))
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = _lbf.lbf_create(p, self.workspace.data_ptr(), nbytes)
        self.N = nx * ny * nz

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            try:
                _lbf.lbf_destroy(ctx)
            except Exception:
                pass
            self.ctx = None

    # -- state -----------------------------------------------------------------------------
    def set_moments(self, M, phi=None):
        """M: (10, nz, ny, nx) float64/float32, CPU or CUDA (public layout)."""
        M = M.contiguous()
        if tuple(M.shape) != (10,) + self.shape:
            raise ValueError(f"moments must have shape {(10,) + self.shape}")
        keep = [M]
        phi_ptr = None
        if phi is not None:
            phi = phi.to(dtype=M.dtype, device=M.device).contiguous()
            keep.append(phi)
            phi_ptr = phi.data_ptr()
        _lbf.lbf_set_moments(self.ctx, M.data_ptr(), _dtype_code(M.dtype), phi_ptr)
        if M.device.type == "cpu":
            # a host source may be read asynchronously (pinned memory): keep it alive until done
            self.stream.synchronize()
        return keep

    def moments(self, dtype=torch.float64, device=None, out=None, phi_out=None):
        """Public state (10, nz, ny, nx) in dtype on `device` (default: the solver's GPU)."""
        if out is None:
            out = torch.empty((10,) + self.shape, dtype=dtype, device=device or self.device)
        phi_ptr = phi_out.data_ptr() if phi_out is not None else None
        _lbf.lbf_moments(self.ctx, out.data_ptr(), _dtype_code(out.dtype), phi_ptr)
        if out.device.type == "cpu":
            self.stream.synchronize()
        return out

    def phi(self, dtype=torch.float64):
        M = torch.empty((10,) + self.shape, dtype=dtype, device=self.device)
        ph = torch.empty(self.shape, dtype=dtype, device=self.device)
        _lbf.lbf_moments(self.ctx, M.data_ptr(), _dtype_code(dtype), ph.data_ptr())
        return ph

    def step(self, n=1):
        _lbf.lbf_step(self.ctx, int(n))

    def reduce(self):
        """[sum p*, sum ux, sum uy, sum uz, sum phi, sum u.u] over fluid sites (FP64)."""
        return _lbf.lbf_reduce(self.ctx)

    def reduce_async(self, out=None):
        """The sums of reduce() copied into `out` (6 float64: a CUDA tensor or pinned host memory,
        default a new pinned host tensor) without waiting; valid once the stream has passed the
        copy (after synchronize()). Step errors surface at the next synchronize() or reduce()."""
        if out is None:
            out = torch.empty(6, dtype=torch.float64).pin_memory()
        if out.dtype != torch.float64 or out.numel() < 6 or not out.is_contiguous():
            raise ValueError("reduce_async needs a contiguous float64 buffer of 6 values")
        _lbf.lbf_reduce_async(self.ctx, out.data_ptr())
        return out

    @property
    def kernels_per_step(self):
        """Kernel launches one step issues (1; 2 with the row split for walls; +2 two components)."""
        return _lbf.lbf_kernels_per_step(self.ctx)

    def synchronize(self):
        _lbf.lbf_synchronize(self.ctx)

    # -- raw internal states (checkpointing, adjoint) ----------------------------------------
    @property
    def state_bytes(self):
        return _lbf.lbf_state_bytes(self.ctx)

    def new_state(self, count=None):
        shape = (self.state_bytes,) if count is None else (count, self.state_bytes)
        return torch.empty(shape, dtype=torch.uint8, device=self.device)

    def copy_state(self, dst):
        _lbf.lbf_copy_state(self.ctx, dst.data_ptr())

    def load_state(self, src):
        _lbf.lbf_load_state(self.ctx, src.data_ptr())

    def step_state(self, src, dst):
        _lbf.lbf_step_state(self.ctx, src.data_ptr(), dst.data_ptr())

    def adjoint_step(self, state_t, state_t1, lam_in, lam_out, grad_force):
        for t, dt in ((lam_in, self.compute_dtype), (lam_out, self.compute_dtype), (grad_force, torch.float64)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError("adjoint buffers: lambda in the compute dtype, grad_force float64, contiguous CUDA")
        _lbf.lbf_adjoint_step(self.ctx, state_t.data_ptr(), state_t1.data_ptr(), lam_in.data_ptr(),
                              lam_out.data_ptr(), grad_force.data_ptr())
