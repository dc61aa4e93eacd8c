"""The C ABI without a GPU: librlb.so builds and loads, exports every entry
point include/rlb.h declares, and validates configurations on the host
(rlb_check_config and the argument checks of rlb_create run before any CUDA
call)."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1302_1125_gb300 import build as B
from paper_1302_1125_gb300 import rlb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rlb.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rlb.lib()


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"RLB_API[^;(]*?\b(rlb_\w+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared()
    for must in ("rlb_create", "rlb_init", "rlb_step", "rlb_macroscopic", "rlb_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", rlb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(rlb_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        assert hasattr(lib, n)


def test_library_does_not_link_the_oracle():
    out = subprocess.run(["nm", "-D", rlb.LIB_PATH], capture_output=True, text=True, check=True).stdout
    assert "orc_" not in out


def cfg(**kw):
    g = dict(nx=64, ny=1, nz=1, bc_lo=(1, 0, 0), bc_hi=(1, 0, 0), inlet=(1.0, 1.0, (0.0, 0.0, 0.0)))
    o = dict(dt_over_dx=0.25)
    for k in list(kw):
        if k in g:
            g[k] = kw.pop(k)
        elif k in ("dt_over_dx", "tau_override", "alpha_override", "euler_mode", "precision", "symmetry_1d",
                   "model", "thread_mapping", "symmetry_2d", "slab_rows"):
            o[k] = kw.pop(k)
    return rlb.make_grid(**g), rlb.make_options(**o), kw


@pytest.mark.parametrize("change,expect", [
    ({}, rlb.RLB_OK),
    ({"Q": 18}, rlb.RLB_E_INVALID),
    ({"nx": 0}, rlb.RLB_E_INVALID),
    ({"nx": 2048, "ny": 2048, "nz": 1024}, rlb.RLB_E_INVALID),
    # the FP32 step addresses a population plane with 32-bit byte offsets
    ({"nx": 1024, "ny": 1024, "nz": 1024, "precision": 1, "dt_over_dx": 0.15}, rlb.RLB_E_INVALID),
    ({"nx": 1024, "ny": 1024, "nz": 1023, "precision": 1, "dt_over_dx": 0.15}, rlb.RLB_OK),
    ({"nx": 1024, "ny": 1024, "nz": 1024, "precision": 0, "dt_over_dx": 0.15}, rlb.RLB_OK),
    ({"eta": -0.1}, rlb.RLB_E_INVALID),
    ({"zeta": math.nan}, rlb.RLB_E_INVALID),
    ({"limiter": 7}, rlb.RLB_E_INVALID),
    ({"precision": 3}, rlb.RLB_E_INVALID),
    ({"bc_lo": (2, 2, 0)}, rlb.RLB_E_INVALID),
    ({"bc_lo": (2, 0, 0), "inlet": (1.0, 1.0, (1.0, 0.0, 0.0))}, rlb.RLB_E_INVALID),
    ({"bc_lo": (2, 0, 0), "inlet": (1.0, 1.0, (0.9, 0.0, 0.0))}, rlb.RLB_OK),
    ({"dt_over_dx": 0.73}, rlb.RLB_E_UNSTABLE),          # 1-D Courant bound 0.72
    ({"dt_over_dx": 0.7}, rlb.RLB_OK),
    ({"ny": 8, "dt_over_dx": 0.37}, rlb.RLB_E_UNSTABLE),  # 2-D bound 0.36
    ({"alpha_override": 1.0}, rlb.RLB_E_UNSTABLE),       # 2 (c0 nu/ct) dt alpha > 1
    ({"alpha_override": 0.5}, rlb.RLB_OK),
    ({"dt_over_dx": -1.0}, rlb.RLB_E_INVALID),
    ({"symmetry_1d": 1}, rlb.RLB_OK),            # a 1-D grid, FP64
    ({"symmetry_1d": 1, "precision": 1}, rlb.RLB_OK),
    ({"symmetry_1d": 1, "precision": 1, "ny": 8}, rlb.RLB_E_INVALID),     # 1-D grids only
    ({"symmetry_1d": 1, "precision": 1, "euler_mode": 1}, rlb.RLB_E_INVALID),
    ({"symmetry_1d": 1, "symmetry_2d": 1, "precision": 1, "ny": 8}, rlb.RLB_E_INVALID),
    ({"symmetry_1d": 1, "precision": 1, "bc_lo": (2, 0, 0),
      "inlet": (1.0, 1.0, (0.5, 0.1, 0.0))}, rlb.RLB_E_INVALID),          # inlet moving in y
    ({"model": 2}, rlb.RLB_E_INVALID),
    ({"thread_mapping": 4}, rlb.RLB_E_INVALID),
    ({"slab_rows": -1}, rlb.RLB_E_INVALID),
    ({"slab_rows": 3, "ny": 64, "nz": 8, "precision": 1, "dt_over_dx": 0.15}, rlb.RLB_OK),
    ({"thread_mapping": 3, "ny": 8, "nz": 8}, rlb.RLB_OK),
    ({"thread_mapping": -1}, rlb.RLB_E_INVALID),
    ({"thread_mapping": 2, "ny": 8, "nz": 8}, rlb.RLB_OK),
    ({"symmetry_2d": 1, "ny": 8, "precision": 1}, rlb.RLB_OK),
    ({"symmetry_2d": 2, "ny": 8, "precision": 1}, rlb.RLB_E_INVALID),
    ({"symmetry_2d": 1, "ny": 8}, rlb.RLB_OK),                              # FP64 too
    ({"symmetry_2d": 1, "ny": 8, "precision": 1, "euler_mode": 1}, rlb.RLB_E_INVALID),
    ({"symmetry_2d": 1, "precision": 1}, rlb.RLB_E_INVALID),                # 1-D grid
    ({"symmetry_2d": 1, "ny": 8, "nz": 4, "precision": 1}, rlb.RLB_E_INVALID),   # 3-D grid
    ({"symmetry_2d": 1, "ny": 8, "precision": 1, "bc_lo": (2, 0, 0),
      "inlet": (1.0, 1.0, (0.5, 0.0, 0.1))}, rlb.RLB_E_INVALID),            # inlet moving in z
    ({"symmetry_2d": 1, "ny": 8, "precision": 1, "bc_lo": (2, 0, 0),
      "inlet": (1.0, 1.0, (0.5, 0.3, 0.0))}, rlb.RLB_OK),
    ({"model": 1, "dt_over_dx": 1.19}, rlb.RLB_OK),        # basic lattice, 1-D: bound sqrt(27/19) = 1.192
    ({"model": 1, "dt_over_dx": 1.2}, rlb.RLB_E_UNSTABLE),
    ({"model": 1, "ny": 8, "dt_over_dx": 0.59}, rlb.RLB_OK),   # 2-D: unit diagonals, bound 0.596
    ({"model": 1, "ny": 8, "dt_over_dx": 0.6}, rlb.RLB_E_UNSTABLE),
])
def test_host_validation(lib, change, expect):
    change = dict(change)
    Q = change.pop("Q", 19)
    eta = change.pop("eta", 0.1)
    zeta = change.pop("zeta", 0.0)
    limiter = change.pop("limiter", 0)
    g, o, rest = cfg(**change)
    assert not rest
    assert rlb.rlb_check_config(g, Q, eta, zeta, limiter, o) == expect
    if expect != rlb.RLB_OK:
        # rlb_create rejects the same configuration before touching the GPU
        with pytest.raises(rlb.RLBError) as e:
            rlb.rlb_create(g, Q, eta, zeta, limiter, o)
        assert e.value.status == expect
        assert rlb.last_error() != ""


def test_status_strings(lib):
    assert rlb.status_string(rlb.RLB_E_NONPHYSICAL) == "RLB_E_NONPHYSICAL"
    assert rlb.status_string(12345) == "RLB_E_UNKNOWN"


def test_null_handles_are_rejected(lib):
    L = rlb.lib()
    assert L.rlb_step(None, 1) == rlb.RLB_E_INVALID
    assert L.rlb_init(None, None, None, None, None, None, 0) == rlb.RLB_E_INVALID
    assert L.rlb_state_bytes(None) == 0
    L.rlb_destroy(None)


def test_struct_layouts_match_the_header(tmp_path):
    """every field of the binding's ctypes structures sits at the offset, and
    every structure has the size, that a C compiler gives the header's"""
    structs = {"rlb_grid": rlb.rlb_grid, "rlb_options": rlb.rlb_options,
               "rlb_batch_tuning": rlb.rlb_batch_tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rlb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for ln in filter(None, out):
        name, field, value = ln.split()
        cls = structs[name]
        expect = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert int(value) == expect, (name, field)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def _prototypes():
    """{name: (return type, [parameter types])} of the header's entry points"""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"RLB_API\s+([^;(]*?)\s*\b(rlb_\w+)\s*\(([^)]*)\)\s*;", src, re.S):
        ps = [" ".join(p.split()) for p in params.split(",")]
        ps = [] if ps == ["void"] else ps
        out[name] = (" ".join(ret.split()), ps)
    return out


_SCALARS = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
            "size_t": ctypes.c_size_t, "rlb_status": ctypes.c_int, "unsigned char": ctypes.c_ubyte,
            "char": ctypes.c_char, "rlb_grid": rlb.rlb_grid, "rlb_options": rlb.rlb_options,
            "rlb_batch_tuning": rlb.rlb_batch_tuning,
            "rlb_ctx *": ctypes.c_void_p, "rlb_batch *": ctypes.c_void_p}   # opaque handles


def _ctype_matches(c_decl, ct):
    """a C declaration ("const double *out", "long long n") against a ctypes
    type: scalars exactly; a pointer as c_void_p (opaque or untyped), or as
    POINTER of the pointee's type"""
    t = re.sub(r"\b(const|restrict)\b", "", c_decl).strip()
    if not t.endswith("*"):
        t = re.sub(r"\s*\w+$", "", t)
    t = " ".join(t.replace("*", " * ").split())
    if t.endswith("*"):
        base = t[:-1].strip()
        if ct is ctypes.c_void_p:
            return True
        if ct is ctypes.c_char_p:
            return base == "char"
        return (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)
                and _SCALARS.get(base) is ct._type_)
    return _SCALARS.get(t) is ct


def test_binding_signatures_match_the_header(lib):
    protos = _prototypes()
    assert sorted(protos) == declared()
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(params), (name, params)
        for decl, ct in zip(params, fn.argtypes):
            assert _ctype_matches(decl, ct), (name, decl, ct)
        if ret == "void":
            assert fn.restype is None, name
        else:
            assert _ctype_matches(ret + " r", fn.restype), (name, ret, fn.restype)


def test_no_gpu_means_an_error_not_a_fallback(lib):
    """without a CUDA device the library reports RLB_E_CUDA for a valid
    configuration: there is no CPU path to fall back on"""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(rlb.RLBError) as e:
        rlb.Grid(16)
    assert e.value.status == rlb.RLB_E_CUDA
    with pytest.raises(rlb.RLBError) as e:
        rlb.Batch([64, 32], [0.1, 0.1], [0.0, 0.0])
    assert e.value.status == rlb.RLB_E_CUDA


def test_a_c_program_uses_the_abi(lib, tmp_path):
    """tests/c/shock_tube.c builds against include/rlb.h and librlb.so with a
    plain C compiler and runs: the host-side check passes, and without a GPU
    rlb_create reports RLB_E_CUDA, which the program prints before it exits 0"""
    exe = tmp_path / "shock_tube"
    libdir = os.path.dirname(rlb.LIB_PATH)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "c", "shock_tube.c"),
                    "-L", libdir, "-l:librlb.so", f"-Wl,-rpath,{libdir}", "-lm"], check=True)
    torch = pytest.importorskip("torch")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    if not torch.cuda.is_available():
        assert r.stdout.startswith("no CUDA device: RLB_E_CUDA"), r.stdout
    else:
        # the gas at the membrane moves at the exact plateau velocity, 0.191
        ux = float(r.stdout.split("u_x at the membrane:")[1].split()[0])
        assert abs(ux - 0.191) < 0.005, r.stdout


def test_state_buffers_are_checked_before_the_library_sees_them():
    """the binding refuses a short or non-contiguous checkpoint buffer
    instead of letting rlb_get_state write past its end"""
    ok = np.zeros(43 * 10, np.float32)
    assert rlb._state_buffer(ok, ok.nbytes) == ok.ctypes.data
    with pytest.raises(ValueError, match="holds"):
        rlb._state_buffer(np.zeros(43 * 10 - 1, np.float32), ok.nbytes)
    with pytest.raises(ValueError, match="contiguous"):
        rlb._state_buffer(np.zeros(2 * 43 * 10, np.float32)[::2], ok.nbytes)
    torch = pytest.importorskip("torch")
    t = torch.zeros(43 * 10, dtype=torch.float32)
    assert rlb._state_buffer(t, ok.nbytes) == t.data_ptr()
    with pytest.raises(ValueError, match="holds"):
        rlb._state_buffer(t[:-1], ok.nbytes)
