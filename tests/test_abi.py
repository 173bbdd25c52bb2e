"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2104_12570_gb300 as hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hpscd_\w+)\s*\(", src, re.M):
            names.add(mt.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("hpscd_create", "hpscd_destroy", "hpscd_solve", "hpscd_solve_host",
                 "hpscd_status_string", "hpscd_workspace_size", "hpscd_set_workspace"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = hp.load()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared but not exported"
        assert name in hp.SIGNATURES, f"{name} has no Python binding"


def test_library_is_built_for_sm_103a_only():
    """Every compile and the link name exactly one target, sm_103a (read from the
    command lines the build records beside the library)."""
    import json
    from paper_2104_12570_gb300 import build
    hp.load()
    info = json.load(open(build.INFO))
    for cmd in info["compile"] + [info["link"]]:
        targets = [cmd[i + 1] for i, a in enumerate(cmd) if a == "-gencode"]
        assert targets == ["arch=compute_103a,code=sm_103a"], cmd
        assert not any(a.startswith(("-arch", "--gpu-architecture")) for a in cmd), cmd


def test_status_strings_and_null_context():
    lib = hp.load()
    assert lib.hpscd_status_string(0) == b"ok"
    assert lib.hpscd_status_string(2).startswith(b"not converged")
    assert lib.hpscd_status_string(99) == b"unknown status"
    o = hp.make_opts()
    rc = lib.hpscd_solve(None, None, 0, 0, 10, 10, 10, None, None, 0, ctypes.byref(o), None,
                         None, None)
    assert rc == 1
    assert lib.hpscd_destroy(None) == 0


def test_layout_detection():
    import numpy as np
    Xc = np.zeros((5, 7), dtype=np.float32).T  # (7, 5) logical, column-major
    _, dt, lay, m, n, ld = hp._describe(Xc)
    assert (dt, lay, m, n, ld) == (hp.F32, hp.COL, 7, 5, 7)
    Xr = np.zeros((7, 5), dtype=np.uint16)
    _, dt, lay, m, n, ld = hp._describe(Xr)
    assert (dt, lay, m, n, ld) == (hp.BF16, hp.ROW, 7, 5, 5)
    with pytest.raises(TypeError):
        hp._describe(np.zeros((3, 3), dtype=np.float64))


def test_every_entry_point_refuses_null_handles():
    """With null handles and pointers (and zero sizes) every entry point returns
    HPSCD_ERR_INVALID_ARG without touching a device; the destroy calls accept NULL."""
    lib = hp.load()
    destroy = {"hpscd_destroy", "hpscd_batch_destroy", "hpscd_mlp_destroy"}
    for name, (args, _) in sorted(hp.SIGNATURES.items()):
        if name in ("hpscd_status_string", "hpscd_mlp_param_count"):
            continue
        vals = [0 if a in (ctypes.c_int, ctypes.c_int64, ctypes.c_size_t)
                else 0.0 if a in (ctypes.c_double, ctypes.c_float) else None for a in args]
        rc = getattr(lib, name)(*vals)
        assert rc == (0 if name in destroy else 1), (name, rc)
    assert lib.hpscd_mlp_param_count() > 0
