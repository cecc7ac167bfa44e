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


def test_size_and_index_validation_without_device():
    """Every check below returns before the library touches the device: meshes past int32
    indexing, empty meshes, and restriction / vertex indices out of range or leaving a DoF
    without an element."""
    import ctypes

    import paper_1910_03032_b300 as hx
    lib, out = hx._lib, ctypes.c_void_p()
    V = np.zeros((8, 3))
    vp = ctypes.c_void_p(V.ctypes.data)
    # (p+1)^3 x elements >= 2^31: rejected before the vertex array is read
    assert lib.hx_mesh_create_box(1024, 1024, 1024, 8, 10, vp, 63, ctypes.byref(out)) == hx.HX_ERR_UNSUPPORTED
    assert lib.hx_mesh_create_box(700, 700, 700, 5, 7, vp, 0, ctypes.byref(out)) == hx.HX_ERR_UNSUPPORTED
    assert "int32" in hx.hx_last_error()
    EV = np.zeros((1, 8), np.int64)
    R1 = np.zeros((1, 8), np.int64)
    ev, r1 = ctypes.c_void_p(EV.ctypes.data), ctypes.c_void_p(R1.ctypes.data)
    assert lib.hx_mesh_create(1, 3, 8, vp, 1 << 29, ev, 8, r1, None, ctypes.byref(out)) == hx.HX_ERR_UNSUPPORTED
    assert lib.hx_mesh_create(1, 3, 8, vp, 1, ev, 1 << 31, r1, None, ctypes.byref(out)) == hx.HX_ERR_UNSUPPORTED
    # empty meshes and missing arrays
    assert lib.hx_mesh_create(1, 3, 8, vp, 0, ev, 8, r1, None, ctypes.byref(out)) == hx.HX_ERR_ARG
    assert lib.hx_mesh_create(1, 3, 8, vp, 1, ev, 0, r1, None, ctypes.byref(out)) == hx.HX_ERR_ARG
    assert lib.hx_mesh_create(1, 3, 8, None, 1, ev, 8, r1, None, ctypes.byref(out)) == hx.HX_ERR_ARG
    assert not out.value
    ev8 = np.arange(8, dtype=np.int64)[None]
    for R, EVx, msg in [(np.array([[0, 1, 2, 3, 4, 5, 6, 8]]), ev8, "outside"),       # DoF id >= n_dof
                        (np.array([[0, 1, 2, 3, 4, 5, 6, -1]]), ev8, "outside"),      # negative DoF id
                        (np.array([[0, 1, 2, 3, 4, 5, 6, 6]]), ev8, "no element"),    # DoF 7 unused
                        (np.arange(8)[None], np.array([[0, 1, 2, 3, 4, 5, 6, 8]]), "elem_vert")]:
        with pytest.raises(hx.HxError) as ei:
            hx.hx_mesh_create(1, 3, V, EVx, 8, R)
        assert ei.value.status == hx.HX_ERR_ARG and msg in hx.hx_last_error()
    # NULL handles and bad counts on the operator, solver and batch entry points
    assert lib.hx_op_create(None, ctypes.c_double(1.0), ctypes.c_double(1.0), None, 0, None,
                            ctypes.byref(out)) == hx.HX_ERR_ARG
    assert lib.hx_batch_create(0, None, None, None, ctypes.c_double(1e-10), 10, 0, ctypes.byref(out)) == hx.HX_ERR_ARG
    for name, args in [("hx_op_set_f32_kernel", (0,)), ("hx_op_set_f32_tile", (0,)), ("hx_op_set_wait_limit", (1,)),
                       ("hx_op_set_coefficients", (ctypes.c_double(1.0), ctypes.c_double(1.0), None, None))]:
        assert getattr(lib, name)(None, *args) == hx.HX_ERR_ARG, name


def test_build_flags_target_sm_103a():
    src = open(os.path.join(ROOT, "paper_1910_03032_b300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src
