"""Host-side checks of the C-ABI library that need no GPU.

* libelbm.so builds for sm_103a, loads, and exports every function that
  include/elbm.h declares (and the Python binding wraps each under its C name);
* the pure host functions (defaults, buffer size) and the argument validation of
  elbm_create return the documented status codes before touching CUDA;
* the product path (package sources, C sources) never names the oracle.
No compute call is made here.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2203_12946_gb300 import build as B
from paper_2203_12946_gb300 import elbm as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "elbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(elbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return E.load()


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 15
    raw = ctypes.CDLL(B.LIB)
    for n in names:
        assert hasattr(raw, n), f"{n} declared in elbm.h but not exported"
        assert hasattr(E, n), f"{n} has no Python binding"
    assert sorted(E.EXPORTED) == names


def test_header_compiles_as_c(tmp_path):
    """The public header is plain C (no C++ or CUDA types in the signatures)."""
    c = tmp_path / "t.c"
    c.write_text('#include "elbm.h"\nint main(void){elbm_opts o; elbm_default_opts(&o); return o.cutoff - 1;}\n')
    import subprocess
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                        os.path.dirname(HEADER), str(c)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_default_opts(lib):
    o = E.elbm_default_opts()
    assert (o.storage, o.alpha_mode, o.cutoff, o.b_variant, o.device, o.rho0) == (
        E.ELBM_STORE_F32, E.ELBM_ALPHA_HIGHER, 1, E.ELBM_B_DERIVED, 0, 1.0)
    assert o.stream is None


@pytest.mark.parametrize("lattice,dims,storage,want", [
    (E.ELBM_D2Q9, (64, 64, 1), E.ELBM_STORE_F64, 9 * 64 * 64 * 8),
    (E.ELBM_D3Q27, (256, 256, 256), E.ELBM_STORE_F32, 27 * 256 ** 3 * 4),
    (E.ELBM_D3Q27, (13, 11, 7), E.ELBM_STORE_F16DEV, 27 * 13 * 11 * 7 * 2),
    (E.ELBM_D2Q9, (1024, 1024, 1), E.ELBM_STORE_BF16DEV, 9 * 1024 * 1024 * 2),
])
def test_population_bytes(lib, lattice, dims, storage, want):
    assert E.elbm_population_bytes(lattice, dims, storage) == want


@pytest.mark.parametrize("lattice,dims,beta,bc,code", [
    (10, (8, 8, 1), 0.9, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D2Q9, (8, 8, 2), 0.9, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D2Q9, (0, 8, 1), 0.9, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, (8, -1, 8), 0.9, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, (8, 8, 8), 1.0, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, (8, 8, 8), 0.0, 0, E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, (8, 8, 8), float("nan"), 0, E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, (8, 8, 8), 0.9, 1, E.ELBM_ERR_UNSUPPORTED),
])
def test_create_rejects_bad_arguments(lib, lattice, dims, beta, bc, code):
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_create(lattice, dims, beta, bc)
    assert ei.value.code == code
    assert "elbm_create" in E.elbm_last_error(None)


@pytest.mark.parametrize("field,value", [("storage", 7), ("alpha_mode", 5), ("b_variant", 2),
                                         ("cutoff", 3), ("rho0", -1.0)])
def test_create_rejects_bad_options(lib, field, value):
    o = E.elbm_default_opts()
    setattr(o, field, value)
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_create(E.ELBM_D2Q9, (8, 8, 1), 0.9, 0, o)
    assert ei.value.code == E.ELBM_ERR_ARG


def test_null_handle_calls_fail_cleanly(lib):
    for fn, args in [(lib.elbm_step, (None, 1)), (lib.elbm_synchronize, (None,)),
                     (lib.elbm_moments, (None, None, None, 0)),
                     (lib.elbm_bind_buffers, (None, None, None, 0))]:
        assert fn(*args) == E.ELBM_ERR_ARG
    lib.elbm_destroy(None)  # safe on NULL
    out = ctypes.c_void_p(None)
    assert lib.elbm_create(None, 9, (ctypes.c_int64 * 3)(8, 8, 1), 0.9, 0, None) == E.ELBM_ERR_ARG
    assert lib.elbm_population_bytes(9, None, 0, None) == E.ELBM_ERR_ARG
    del out


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2203_12946_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"(^|\n)\s*(import|from)\s+oracle\b|elbm_oracle|\bor_[a-z_]+\(",
                                     txt), f"{fn} imports or calls the oracle"
    assert "oracle" not in open(HEADER).read()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """With no built library and no way to build it, loading raises instead of falling back."""
    monkeypatch.setattr(B, "LIB", str(tmp_path / "libelbm.so"))
    monkeypatch.setattr(E, "_lib", None)
    with pytest.raises(ImportError):
        E.load(build_if_missing=False)
    monkeypatch.setattr(E, "_lib", None)


@pytest.mark.parametrize("lattice,dims,betas,code", [
    (8, [(8, 8, 1)], [0.9], E.ELBM_ERR_ARG),
    (E.ELBM_D2Q9, [], [], E.ELBM_ERR_ARG),
    (E.ELBM_D2Q9, [(8, 8, 2)], [0.9], E.ELBM_ERR_ARG),
    (E.ELBM_D2Q9, [(8, 8, 1), (0, 8, 1)], [0.9, 0.9], E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, [(8, 8, 8), (70000, 2, 2)], [0.9, 0.9], E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, [(8, 8, 8), (4, 4, 4)], [0.9, 1.0], E.ELBM_ERR_ARG),
    (E.ELBM_D3Q27, [(8, 8, 8), (2048, 2048, 64)], [0.9, 0.9], E.ELBM_ERR_UNSUPPORTED),
])
def test_batch_create_rejects_bad_arguments(lib, lattice, dims, betas, code):
    with pytest.raises(E.ElbmError) as ei:
        E.elbm_batch_create(lattice, dims, betas)
    assert ei.value.code == code
    assert "elbm_batch_create" in E.elbm_batch_last_error(None)


def test_binding_constants_match_the_header():
    """Every #define ELBM_* integer constant of include/elbm.h has the same value in the
    Python binding (which marshals arguments only and must not drift from the C ABI)."""
    import re

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "elbm.h")).read()
    defs = dict(re.findall(r"#define\s+(ELBM_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", hdr))
    assert len(defs) > 20
    for name, value in defs.items():
        assert getattr(E, name, None) == int(value), name


def test_struct_layouts_match_the_binding(tmp_path):
    """elbm_opts and elbm_diag as the C compiler lays them out (size and every field's
    offset) equal the ctypes mirrors the binding passes by pointer."""
    import subprocess

    structs = {"elbm_opts": E.elbm_opts, "elbm_diag": E.elbm_diag}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "elbm.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0;}")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for sname, cls in structs.items():
        assert got[(sname, "size")] == ctypes.sizeof(cls), sname
        for fname, _ in cls._fields_:
            assert got[(sname, fname)] == getattr(cls, fname).offset, (sname, fname)


def test_noalloc_rejects_wrapping_dims_and_misaligned_buffers_before_cuda(lib):
    """elbm_diagnostics_noalloc decides its argument errors on the host before any CUDA
    call (so they come back as ELBM_ERR_ARG here, without a GPU): sides of up to 2^30 whose
    product wraps around in 64 bits (2^30 * 2^30 * 2^4 = 2^64 reads as 0, * 2^5 as 2) are
    more than 2^31 nodes, and a buffer address that is not a multiple of the element size
    is refused before it could be read."""
    fn = lib.elbm_diagnostics_noalloc
    d = E.elbm_diag()
    opts = E.elbm_default_opts()
    for dims in ((1 << 30, 1 << 30, 1 << 4), (1 << 30, 1 << 30, 1 << 5), (1 << 30, 1 << 2, 1 << 30)):
        code = fn(E.ELBM_D3Q27, E._dims(dims), 0.9, ctypes.byref(opts), 4096, ctypes.byref(d), None)
        assert code == E.ELBM_ERR_ARG and "2^31" in E.elbm_last_error(None)
    for storage, addr in ((E.ELBM_STORE_F32, 4098), (E.ELBM_STORE_F64, 4100), (E.ELBM_STORE_F16DEV, 4097)):
        opts.storage = storage
        code = fn(E.ELBM_D2Q9, E._dims((8, 8, 1)), 0.9, ctypes.byref(opts), addr, ctypes.byref(d), None)
        assert code == E.ELBM_ERR_ARG and "aligned" in E.elbm_last_error(None)
