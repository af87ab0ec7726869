"""ctypes binding of the C ABI in include/lbf.h: one Python function per C entry point, same
names, argument marshalling only. Every non-OK status raises LBFError with the library's own
message. There is no fallback: if liblbf.so is missing or cannot be loaded this module raises."""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBF_LIBRARY selects another build of the same library (e.g. the index-checked liblbf_debug.so)
LIB_PATH = os.environ.get("LBF_LIBRARY") or os.path.join(_PKG, "liblbf.so")

LBF_D3Q19, LBF_D3Q27, LBF_D3Q27H = 19, 27, 127
LBF_F64, LBF_F32, LBF_F16, LBF_BF16 = 0, 1, 2, 3
LBF_OK, LBF_EINVAL, LBF_ENOMEM, LBF_ECUDA, LBF_EUNSTABLE, LBF_EINTERNAL, LBF_ENOTSUP = range(7)
LBF_ROUND_STOCHASTIC, LBF_ROUND_NEAREST = 0, 1

# every symbol declared in include/lbf.h
EXPORTS = ("lbf_workspace_bytes", "lbf_validate", "lbf_create", "lbf_set_moments", "lbf_step", "lbf_moments",
           "lbf_reduce", "lbf_reduce_async", "lbf_synchronize", "lbf_state_bytes", "lbf_copy_state", "lbf_load_state",
           "lbf_step_state", "lbf_adjoint_step", "lbf_step_static", "lbf_destroy", "lbf_status_string",
           "lbf_last_error", "lbf_version", "lbf_kernels_per_step")


class lbf_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("storage", ctypes.c_int), ("tau", ctypes.c_double), ("force", ctypes.c_double * 3),
        ("force_field", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("two_component", ctypes.c_int),
        ("rho_l", ctypes.c_double), ("rho_h", ctypes.c_double), ("tau_l", ctypes.c_double),
        ("tau_h", ctypes.c_double), ("sigma", ctypes.c_double), ("width", ctypes.c_double),
        ("diffusivity", ctypes.c_double), ("scale_hint", ctypes.c_double * 3), ("stream", ctypes.c_void_p),
        ("rounding", ctypes.c_int), ("populations", ctypes.c_int), ("body_accel", ctypes.c_double * 3),
    ]


class LBFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load liblbf.so (built in-tree by paper_2609_09160_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2609_09160_gb300.build` "
                           "(the package has no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, VP, I, SZ, D = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
    sig = {
        "lbf_workspace_bytes": (SZ, [P(lbf_params)]),
        "lbf_validate": (I, [P(lbf_params)]),
        "lbf_create": (I, [P(VP), P(lbf_params), VP, SZ]),
        "lbf_set_moments": (I, [VP, VP, I, VP]),
        "lbf_step": (I, [VP, I]),
        "lbf_moments": (I, [VP, VP, I, VP]),
        "lbf_reduce": (I, [VP, P(D)]),
        "lbf_reduce_async": (I, [VP, VP]),
        "lbf_synchronize": (I, [VP]),
        "lbf_state_bytes": (SZ, [VP]),
        "lbf_copy_state": (I, [VP, VP]),
        "lbf_load_state": (I, [VP, VP]),
        "lbf_step_state": (I, [VP, VP, VP]),
        "lbf_adjoint_step": (I, [VP, VP, VP, VP, VP, VP]),
        "lbf_step_static": (I, [P(lbf_params), VP, VP, VP, VP, VP]),
        "lbf_destroy": (I, [VP]),
        "lbf_status_string": (ctypes.c_char_p, [I]),
        "lbf_last_error": (ctypes.c_char_p, []),
        "lbf_version": (I, []),
        "lbf_kernels_per_step": (I, [VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_name(s):
    return load_library().lbf_status_string(int(s)).decode()


def _check(status):
    if status != LBF_OK:
        raise LBFError(status, load_library().lbf_last_error().decode())


def lbf_workspace_bytes(params):
    return load_library().lbf_workspace_bytes(ctypes.byref(params))


def lbf_validate(params):
    return load_library().lbf_validate(ctypes.byref(params))


def lbf_create(params, workspace_ptr, nbytes):
    ctx = ctypes.c_void_p()
    _check(load_library().lbf_create(ctypes.byref(ctx), ctypes.byref(params), ctypes.c_void_p(workspace_ptr),
                                     nbytes))
    return ctx


def lbf_set_moments(ctx, src_ptr, src_dtype, phi_ptr=None):
    _check(load_library().lbf_set_moments(ctx, ctypes.c_void_p(src_ptr), src_dtype, ctypes.c_void_p(phi_ptr)))


def lbf_step(ctx, n):
    _check(load_library().lbf_step(ctx, n))


def lbf_moments(ctx, dst_ptr, dst_dtype, phi_ptr=None):
    _check(load_library().lbf_moments(ctx, ctypes.c_void_p(dst_ptr), dst_dtype, ctypes.c_void_p(phi_ptr)))


def lbf_reduce(ctx):
    out = (ctypes.c_double * 6)()
    _check(load_library().lbf_reduce(ctx, out))
    return [out[i] for i in range(6)]


def lbf_reduce_async(ctx, dst_ptr):
    _check(load_library().lbf_reduce_async(ctx, ctypes.c_void_p(dst_ptr)))


def lbf_synchronize(ctx):
    _check(load_library().lbf_synchronize(ctx))


def lbf_state_bytes(ctx):
    return load_library().lbf_state_bytes(ctx)


def lbf_copy_state(ctx, dst_ptr):
    _check(load_library().lbf_copy_state(ctx, ctypes.c_void_p(dst_ptr)))


def lbf_load_state(ctx, src_ptr):
    _check(load_library().lbf_load_state(ctx, ctypes.c_void_p(src_ptr)))


def lbf_step_state(ctx, src_ptr, dst_ptr):
    _check(load_library().lbf_step_state(ctx, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr)))


def lbf_adjoint_step(ctx, state_t_ptr, state_t1_ptr, lam_in_ptr, lam_out_ptr, grad_force_ptr):
    _check(load_library().lbf_adjoint_step(ctx, ctypes.c_void_p(state_t_ptr), ctypes.c_void_p(state_t1_ptr),
                                           ctypes.c_void_p(lam_in_ptr), ctypes.c_void_p(lam_out_ptr),
                                           ctypes.c_void_p(grad_force_ptr)))


def lbf_step_static(params, src_ptr, dst_ptr, mask_ptr=None, sums_ptr=None, flags_ptr=None):
    """One step from src to dst with no device allocation (static scratch in the library)."""
    _check(load_library().lbf_step_static(ctypes.byref(params), ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr),
                                          ctypes.c_void_p(mask_ptr), ctypes.c_void_p(sums_ptr),
                                          ctypes.c_void_p(flags_ptr)))


def lbf_debug_wait_probe(ctx, polls):
    """Test hook of the LBF_DEBUG library (include/lbf_debug.h): a bounded mbarrier wait that gives
    up after `polls` polls and sets the context's error flag. Raises if the loaded library is the
    release build, which does not export it."""
    lib = load_library()
    if not hasattr(lib, "lbf_debug_wait_probe"):
        raise RuntimeError("lbf_debug_wait_probe is exported by the LBF_DEBUG build (liblbf_debug.so) only")
    fn = lib.lbf_debug_wait_probe
    fn.restype, fn.argtypes = ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint]
    _check(fn(ctx, polls))


def lbf_destroy(ctx):
    _check(load_library().lbf_destroy(ctx))


def lbf_status_string(status):
    return load_library().lbf_status_string(int(status)).decode()


def lbf_last_error():
    return load_library().lbf_last_error().decode()


def lbf_version():
    return load_library().lbf_version()


def lbf_kernels_per_step(ctx):
    return load_library().lbf_kernels_per_step(ctx)
