"""The C-ABI library builds, loads and exports every symbol include/lbf.h declares; host-only
entry points (validation, workspace layout, status strings) behave as documented. No GPU."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2609_09160_gb300 import _lbf, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lbf.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbf_[a-z_0-9]+)\s*\(", text)))


def test_every_declaration_cites_the_paper_or_says_it_has_no_counterpart():
    """Each function of include/lbf.h carries, in the comment right above it, the passage of the
    paper it implements ("Paper: Eq. ..., Sec. ...") or states that the paper has no counterpart."""
    text = open(os.path.join(ROOT, "include", "lbf.h")).read()
    body = text[text.index("} lbf_params;"):]
    for name in declared_symbols():
        m = re.search(r"/\*((?:(?!\*/).)*)\*/\s*[A-Za-z_][A-Za-z_0-9 *]*\b" + name + r"\s*\(", body, flags=re.S)
        assert m is not None, f"{name}: no comment right above the declaration"
        note = m.group(1)
        assert "Paper:" in note, name
        cited = re.search(r"Paper:.*(Eq\.|Sec\.|no counterpart)", note, flags=re.S)
        assert cited is not None, f"{name}: the comment names no passage"


def test_debug_library_exports_its_test_hooks():
    """liblbf_debug.so (LBF_DEBUG) exports every symbol of include/lbf_debug.h and of lbf.h."""
    dbg = ctypes.CDLL(build.build(debug=True))
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lbf_debug.h")).read(), flags=re.S)
    hooks = sorted(set(re.findall(r"\b(lbf_[a-z_0-9]+)\s*\(", text)))
    assert hooks == ["lbf_debug_wait_probe"]
    for name in hooks + declared_symbols():
        assert ctypes.cast(getattr(dbg, name), ctypes.c_void_p).value, name


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(_lbf.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_struct_layout_matches_the_header(tmp_path):
    """The ctypes lbf_params has the C struct's size and field offsets (compiled with the host C
    compiler against include/lbf.h)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    fields = [f for f, _ in _lbf.lbf_params._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbf.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(lbf_params));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(lbf_params, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(_lbf.lbf_params)] + [getattr(_lbf.lbf_params, f).offset for f in fields]
    assert got == want


def params(**kw):
    p = _lbf.lbf_params()
    p.lattice, p.nx, p.ny, p.nz, p.storage, p.tau = 19, 16, 16, 16, _lbf.LBF_F32, 0.8
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_population_workspace_holds_two_population_buffers(lib):
    """The population representation keeps Q fields per buffer (Sec. 3 memory model: 38 GB for
    D3Q19 and 54 GB for D3Q27 in FP64 at 512^3 for the two buffers) plus one 10-field moment buffer."""
    for lattice in (19, 27):
        p = params(nx=512, ny=512, nz=512, storage=_lbf.LBF_F64, lattice=lattice, populations=1)
        need = _lbf.lbf_workspace_bytes(p)
        pops = 2 * lattice * 512 ** 3 * 8
        assert pops + 10 * 512 ** 3 * 8 <= need < pops + 10 * 512 ** 3 * 8 + 64 * 2 ** 20
        assert pops == {19: 38, 27: 54}[lattice] * 2 ** 30


def test_workspace_holds_two_moment_buffers(lib):
    """Two buffers of 10 fields: the paper's 20 scalar fields per site (Sec. 3 memory model)."""
    for storage, b in ((_lbf.LBF_F64, 8), (_lbf.LBF_F32, 4), (_lbf.LBF_F16, 2), (_lbf.LBF_BF16, 2)):
        p = params(nx=512, ny=512, nz=512, storage=storage)
        need = _lbf.lbf_workspace_bytes(p)
        moments = 20 * 512 ** 3 * b
        assert moments <= need < moments + 64 * 2 ** 20
    # FP64 512^3 moments = 20 GB exactly (GB = 2^30 bytes), as printed in Sec. 3
    assert 20 * 512 ** 3 * 8 == 20 * 2 ** 30


@pytest.mark.parametrize("kw,status", [
    (dict(lattice=15), _lbf.LBF_EINVAL),
    (dict(lattice=28), _lbf.LBF_EINVAL),
    (dict(lattice=_lbf.LBF_D3Q27H, populations=1), _lbf.LBF_ENOTSUP),
    (dict(nx=0), _lbf.LBF_EINVAL),
    (dict(tau=0.5), _lbf.LBF_EINVAL),
    (dict(storage=7), _lbf.LBF_EINVAL),
    (dict(rounding=2), _lbf.LBF_EINVAL),
    (dict(populations=1, storage=_lbf.LBF_F16), _lbf.LBF_ENOTSUP),
    (dict(populations=1, two_component=1, tau_l=1.0, tau_h=1.0, rho_l=1.0, rho_h=1.0, width=4.0, sigma=0.03,
          diffusivity=0.1), _lbf.LBF_ENOTSUP),
    (dict(two_component=1, tau_l=1.0, tau_h=1.0, rho_l=0.5, rho_h=1.5, width=4.0, sigma=0.03, diffusivity=0.1,
          storage=_lbf.LBF_F16), _lbf.LBF_ENOTSUP),
    (dict(body_accel=(0.0, 0.0, 1e-6)), _lbf.LBF_EINVAL),
    (dict(two_component=1, tau_l=1.0, tau_h=0.4, rho_l=1.0, rho_h=1.0, width=4.0, sigma=0.03, diffusivity=0.1),
     _lbf.LBF_EINVAL),
])
def test_validation_rejects_bad_parameters(lib, kw, status):
    p = params(**kw)
    assert _lbf.lbf_validate(p) == status
    assert _lbf.lbf_workspace_bytes(p) == 0
    assert _lbf.lbf_last_error()


def test_valid_parameters(lib):
    assert _lbf.lbf_validate(params()) == _lbf.LBF_OK
    for lattice in (_lbf.LBF_D3Q19, _lbf.LBF_D3Q27, _lbf.LBF_D3Q27H):
        for storage in (_lbf.LBF_F64, _lbf.LBF_F32, _lbf.LBF_F16, _lbf.LBF_BF16):
            assert _lbf.lbf_validate(params(lattice=lattice, storage=storage)) == _lbf.LBF_OK
    # density contrast (FP32/FP64): one more 3-vector field (grad phi) than equal densities
    tc = dict(two_component=1, tau_l=1.0, tau_h=0.8, rho_l=1.0, rho_h=1.0, width=4.0, sigma=0.03, diffusivity=0.1)
    eq = _lbf.lbf_workspace_bytes(params(**tc))
    ctr = _lbf.lbf_workspace_bytes(params(**dict(tc, rho_h=2.0, body_accel=(0.0, 1e-6, 0.0))))
    assert eq > 0 and ctr - eq >= 3 * 16 ** 3 * 4
    # D3Q27h keeps the 10-field state: same workspace as D3Q27
    assert _lbf.lbf_workspace_bytes(params(lattice=_lbf.LBF_D3Q27H)) == _lbf.lbf_workspace_bytes(params(lattice=27))
    tc = params(two_component=1, tau_l=1.0, tau_h=0.8, rho_l=1.0, rho_h=1.0, width=4.0, sigma=0.03, diffusivity=0.1)
    assert _lbf.lbf_validate(tc) == _lbf.LBF_OK


def test_create_rejects_missing_or_small_workspace_before_touching_the_gpu(lib):
    p = params()
    with pytest.raises(_lbf.LBFError) as e:
        _lbf.lbf_create(p, 0, 1 << 30)
    assert e.value.status == _lbf.LBF_EINVAL
    with pytest.raises(_lbf.LBFError) as e:
        _lbf.lbf_create(p, 256, 1024)
    assert e.value.status == _lbf.LBF_ENOMEM
    with pytest.raises(_lbf.LBFError) as e:
        _lbf.lbf_create(p, 4096 + 8, 1 << 40)
    assert e.value.status == _lbf.LBF_ENOMEM


def test_status_strings(lib):
    names = [_lbf.lbf_status_string(s) for s in range(7)]
    assert names == ["LBF_OK", "LBF_EINVAL", "LBF_ENOMEM", "LBF_ECUDA", "LBF_EUNSTABLE", "LBF_EINTERNAL",
                     "LBF_ENOTSUP"]
    assert _lbf.lbf_version() >= 1
