"""The C-ABI library builds, loads and exports every function include/gpmppi.h
declares; argument validation answers with status codes before any GPU work
(no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2411_03289_gb300 as gp
from paper_2411_03289_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "gpmppi.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gp.load()


def test_header_parses():
    names = declared_functions()
    assert "mppi_step" in names and "gp_fit" in names and "mppi_create" in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(gp.EXPORTS) == set(names)


def test_exported_with_c_linkage():
    B.build()
    out = os.popen(f"nm -D --defined-only {B.LIB_PATH}").read()
    for n in declared_functions():
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_version_and_empty_error(lib):
    assert gp.gpmppi_version() == 100
    assert isinstance(gp.gpmppi_last_error(), str)


def test_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    hy = (gp.Hyper * 2)()
    # NULL output handle
    assert lib.gp_fit(None, None, 0, ctypes.cast(hy, ctypes.c_void_p), None) == gp.GPMPPI_ERR_INVALID_ARG
    # N out of range
    assert lib.gp_fit(None, None, -1, ctypes.cast(hy, ctypes.c_void_p), ctypes.byref(h)) == gp.GPMPPI_ERR_INVALID_ARG
    assert lib.gp_fit(None, None, 5000, ctypes.cast(hy, ctypes.c_void_p), ctypes.byref(h)) == gp.GPMPPI_ERR_INVALID_ARG
    assert "N out of range" in gp.gpmppi_last_error()
    # non-finite inputs
    X = np.zeros((3, 4))
    X[1, 2] = np.nan
    Y = np.zeros((3, 2))
    for j in range(2):
        hy[j].lengthscale[:] = [0.5] * 4
        hy[j].signal_var = 0.1
        hy[j].noise_var = 1e-4
    rc = lib.gp_fit(X.ctypes.data_as(ctypes.c_void_p), Y.ctypes.data_as(ctypes.c_void_p), 3,
                    ctypes.cast(hy, ctypes.c_void_p), ctypes.byref(h))
    assert rc == gp.GPMPPI_ERR_NONFINITE
    # bad hyper-parameters
    hy[0].lengthscale[1] = 0.0
    X[1, 2] = 0.0
    rc = lib.gp_fit(X.ctypes.data_as(ctypes.c_void_p), Y.ctypes.data_as(ctypes.c_void_p), 3,
                    ctypes.cast(hy, ctypes.c_void_p), ctypes.byref(h))
    assert rc == gp.GPMPPI_ERR_INVALID_ARG and "lengthscale" in gp.gpmppi_last_error()
    # invalid handles
    assert lib.mppi_step(None, None, None, None, None, None, None) == gp.GPMPPI_ERR_INVALID_ARG
    assert lib.mppi_destroy(None) == gp.GPMPPI_ERR_INVALID_ARG
    assert lib.gp_destroy(None) == gp.GPMPPI_ERR_INVALID_ARG
    assert lib.mppi_create(None, None, 0, None, 0, None, ctypes.byref(h)) == gp.GPMPPI_ERR_INVALID_ARG


def test_struct_layouts_match_header(tmp_path):
    """Compile a C program against the header and compare every field offset
    and struct size with the ctypes mirrors used by the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"gpmppi_params": [f[0] for f in gp.Params._fields_],
              "gpmppi_hyper": [f[0] for f in gp.Hyper._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gpmppi.h"', "int main(void){"]
    for st, names in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for n in names:
            cn = "lambda" if n == "lambda_" else n
            lines.append(f'printf("{st} {n} %zu\\n", offsetof({st}, {cn}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    mirror = {"gpmppi_params": gp.Params, "gpmppi_hyper": gp.Hyper}
    for line in out:
        if not line.strip():
            continue
        st, name, val = line.split()
        cls = mirror[st]
        got = ctypes.sizeof(cls) if name == "size" else getattr(cls, name).offset
        assert got == int(val), (st, name, got, val)


def test_binding_has_no_cpu_fallback(tmp_path, monkeypatch):
    """The binding fails loudly instead of computing anything itself: a
    missing library raises at load(), and host (CPU) tensors are refused
    before any call into the library."""
    import torch
    monkeypatch.setattr(gp, "_lib", None)
    monkeypatch.setattr(gp, "LIB_PATH", str(tmp_path / "libgpmppi_missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gp.load()
    with pytest.raises(ValueError, match="CUDA tensor"):
        gp._dptr(torch.zeros(4), name="U_nom")
