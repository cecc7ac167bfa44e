"""The C-ABI library loads and exports every entry point include/hx.h declares (no GPU needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "hx.h")).read()
    return sorted(set(re.findall(r"^HX_API\s+[\w\s\*]+?\b(hx_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ["hx_mesh_create", "hx_mesh_create_structured", "hx_op_create", "hx_op_apply", "hx_op_diagonal",
              "hx_solve_pcg", "hx_op_destroy", "hx_mesh_destroy", "hx_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1910_03032_b300 as hx
    out = subprocess.run(["nm", "-D", "--defined-only", hx.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(hx_\w+)$", out, flags=re.M))
    assert set(header_functions()) <= exported
    # the binding wraps exactly the declared entry points, under the same names
    assert set(hx.SIGNATURES) == set(header_functions())
    for n in header_functions():
        assert callable(getattr(hx, n))


def test_argument_validation_without_device():
    import paper_1910_03032_b300 as hx
    assert hx.hx_version() >= 100
    V = np.zeros((8, 3))
    for p, q in [(0, 2), (9, 10), (3, 3), (3, 6)]:
        with pytest.raises(hx.HxError) as ei:
            hx.hx_mesh_create_structured(1, 1, 1, p, q, V)
        assert ei.value.status == hx.HX_ERR_UNSUPPORTED
        assert "p" in hx.hx_last_error() or "q" in hx.hx_last_error()
    with pytest.raises(hx.HxError) as ei:
        hx.hx_mesh_create_structured(0, 1, 1, 2, 4, np.zeros((4, 3)))
    assert ei.value.status == hx.HX_ERR_ARG


def test_build_flags_target_sm_103a():
    src = open(os.path.join(ROOT, "paper_1910_03032_b300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
