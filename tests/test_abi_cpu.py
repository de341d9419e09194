"""The C-ABI library builds for sm_103a, loads, and exports every entry point declared in
include/rpa.h.  No GPU needed (no compute calls)."""
import ctypes as C
import re

import numpy as np

import paper_2609_16408_gb300 as R


def test_library_exports_every_declared_symbol():
    lib = R.load()
    declared = R.header_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name


def test_header_functions_are_extern_c_and_documented():
    import os
    txt = open(os.path.join(os.path.dirname(R.__file__), "..", "include", "rpa.h")).read()
    assert 'extern "C"' in txt
    # every declaration carries a comment block right above it or on the same group
    for name in R.header_symbols():
        assert re.search(r"\b" + name + r"\s*\(", txt)


def test_status_strings_and_defaults_without_gpu():
    lib = R.load()
    for st in range(9):
        s = lib.rpa_status_string(st)
        assert isinstance(s, bytes) and len(s) > 0
    o = R.rpa_default_options()
    assert o.lanczos_max == 20 and o.reorth == 1 and o.precision == R.RPA_FP64
    assert list(o.stride) == [1, 1, 1]


def test_invalid_arguments_rejected_on_host():
    lib = R.load()
    # null output pointer / null grid are rejected before any CUDA call
    assert lib.rpa_create(None, None, None) == R.RPA_EINVAL
    g = R.Grid()
    g.n[:] = [0, 4, 4]
    g.h[:] = [0.5, 0.5, 0.5]
    g.bc[:] = [0, 0, 0]
    g.fd_radius = 6
    out = C.c_void_p()
    assert lib.rpa_create(C.byref(out), C.byref(g), None) == R.RPA_EINVAL
    g.n[:] = [4, 4, 4]
    g.fd_radius = 9
    assert lib.rpa_create(C.byref(out), C.byref(g), None) == R.RPA_EINVAL
    assert lib.rpa_tridiag_f11(1, 0, None, None, 0, None) == R.RPA_EINVAL
    assert lib.rpa_gl_frequencies(0, None, None) == R.RPA_EINVAL


def test_ctypes_structs_match_the_c_header(tmp_path):
    """The binding's Grid / Options / Stats mirror rpa_grid / rpa_options / rpa_stats field by
    field: sizes and offsets from a host C compilation of include/rpa.h."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no host C compiler")
    inc = os.path.join(os.path.dirname(R.__file__), "..", "include")
    structs = {"rpa_grid": R.Grid, "rpa_options": R.Options, "rpa_stats": R.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rpa.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-x", "c", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            cname, key, val = ln.split()
            got[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_argument_counts_match_prototypes():
    """Every declared entry point is bound with as many arguments as its C prototype."""
    import os
    txt = open(os.path.join(os.path.dirname(R.__file__), "..", "include", "rpa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    lib = R.load()
    for name in R.header_symbols():
        m = re.search(r"\b" + name + r"\s*\(([^)]*)\)\s*;", txt)
        assert m, name
        params = [p for p in m.group(1).split(",") if p.strip() and p.strip() != "void"]
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue  # not called through the binding
        assert len(fn.argtypes) == len(params), (name, len(fn.argtypes), len(params))
