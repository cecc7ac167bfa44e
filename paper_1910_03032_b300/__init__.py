"""Python binding of libhx.so: the B300 matrix-free Q_p Helmholtz operator and Jacobi-PCG.

Argument marshalling only.  Every computation runs in the CUDA library
behind ``include/hx.h``; the functions here carry the same names as its C
entry points, take torch CUDA tensors (float64, contiguous) for device
buffers and numpy arrays / CPU tensors for host buffers, check their sizes,
and raise ``HxError`` when the library returns a non-zero status.  The
library must be built first (``python paper_1910_03032_b300/build.py``);
importing without it raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhx.so")

HX_OK = 0
HX_ERR_ARG = -1
HX_ERR_CUDA = -2
HX_ERR_OOM = -3
HX_ERR_INVALID_MESH = -4
HX_ERR_NOT_CONVERGED = -5
HX_ERR_BREAKDOWN = -6
HX_ERR_UNSUPPORTED = -7
HX_GEOM_STORED = 0
HX_GEOM_ONTHEFLY = 1
HX_PREC_JACOBI = 0
HX_PREC_COLLOCATED_MASS = 1
HX_PREC_LOR = 2
HX_PREC_LOR_MC = 3
HX_PREC_LOR_MG = 4

_NAMES = {0: "HX_OK", -1: "HX_ERR_ARG", -2: "HX_ERR_CUDA", -3: "HX_ERR_OOM", -4: "HX_ERR_INVALID_MESH",
          -5: "HX_ERR_NOT_CONVERGED", -6: "HX_ERR_BREAKDOWN", -7: "HX_ERR_UNSUPPORTED"}

_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("b_norm", ctypes.c_double),
                ("kernel_launches", ctypes.c_int), ("refinements", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_SIZES = [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I), ctypes.POINTER(_I)]

# Every entry point of include/hx.h: name -> (restype, argtypes)
SIGNATURES = {
    "hx_version": (ctypes.c_int, []),
    "hx_last_error": (ctypes.c_char_p, []),
    "hx_mesh_create": (_I, [_I, _I, _I64, _P, _I64, _P, _I64, _P, _P, ctypes.POINTER(_P)]),
    "hx_mesh_create_structured": (_I, [_I, _I, _I, _I, _I, _P, ctypes.POINTER(_P)]),
    "hx_mesh_create_box": (_I, [_I, _I, _I, _I, _I, _P, _I, ctypes.POINTER(_P)]),
    "hx_mesh_destroy": (None, [_P]),
    "hx_mesh_info": (_I, _SIZES),
    "hx_mesh_qpoint_coords": (_I, [_P, _P, _P]),
    "hx_mesh_node_coords": (_I, [_P, _P, _P]),
    "hx_op_create": (_I, [_P, _D, _D, _P, _I, _P, ctypes.POINTER(_P)]),
    "hx_op_info": (_I, _SIZES),
    "hx_op_set_coefficients": (_I, [_P, _D, _D, _P, _P]),
    "hx_op_launch_count": (ctypes.c_int64, [_P]),
    "hx_op_destroy": (None, [_P]),
    "hx_op_apply": (_I, [_P, _P, _P, _I, _P]),
    "hx_op_diagonal": (_I, [_P, _P, _I, _P]),
    "hx_op_load_vector": (_I, [_P, _P, _P, _P]),
    "hx_solve_pcg": (_I, [_P, _P, _P, _D, _I, _I, _P, ctypes.POINTER(SolveInfo)]),
    "hx_solve_pcg_host": (_I, [_P, _P, _P, _D, _I, _I, _P, ctypes.POINTER(SolveInfo)]),
    "hx_solve_pcg_mixed": (_I, [_P, _P, _P, _D, _I, _D, _P, ctypes.POINTER(SolveInfo)]),
    "hx_op_apply_f32": (_I, [_P, _P, _P, _P]),
    "hx_op_set_wait_limit": (_I, [_P, _I]),
    "hx_op_set_f32_kernel": (_I, [_P, _I]),
    "hx_op_set_f32_tile": (_I, [_P, _I]),
    "hx_op_f32_kernel": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "hx_op_gradient": (_I, [_P, _P, _P, _P, _P, _P]),
    "hx_op_collocated_mass": (_I, [_P, _P, _P]),
    "hx_op_set_preconditioner": (_I, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "hx_op_lor_csr": (_I, [_P, ctypes.POINTER(ctypes.c_int64), _P, _P, _P, _P]),
    "hx_op_precond_apply": (_I, [_P, _P, _P, _P]),
    "hx_batch_create": (_I, [_I, _P, _P, _P, _D, _I, _I, ctypes.POINTER(_P)]),
    "hx_batch_solve": (_I, [_P, _P, _P]),
    "hx_batch_lanes": (_I, [_P]),
    "hx_batch_destroy": (None, [_P]),
    "hx_probe_fma": (_I, [_I, _I64, _P, ctypes.POINTER(_D)]),
    "hx_apply_noalloc": (_I, [_I, _I, _I64, _I64, _P, _P, _P, _P, _D, _D, _P, _P, _P]),
}

HX_NOALLOC_MAX_EVEC = 1 << 22


class HxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_NAMES.get(status, status)}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python paper_1910_03032_b300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status: int) -> int:
    if status != HX_OK:
        raise HxError(status, _lib.hx_last_error().decode())
    return status


def _dptr(t, n=None, name="tensor"):
    """Device pointer of a contiguous float64 CUDA tensor with n elements."""
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float64")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, n, name="array"):
    """Host pointer of a contiguous float64 numpy array or CPU tensor with n elements."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise TypeError(f"{name} must be a contiguous float64 CPU tensor")
        if a.numel() != n:
            raise ValueError(f"{name} has {a.numel()} elements, expected {n}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous float64 numpy array")
    if a.size != n:
        raise ValueError(f"{name} has {a.size} elements, expected {n}")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def hx_version() -> int:
    return _lib.hx_version()


def hx_last_error() -> str:
    return _lib.hx_last_error().decode()


def hx_mesh_create(p, q, vert_xyz, elem_vert, n_dof, restriction, dirichlet=None):
    vert_xyz = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    elem_vert = np.ascontiguousarray(elem_vert, dtype=np.int64)
    restriction = np.ascontiguousarray(restriction, dtype=np.int64)
    n_elem = elem_vert.shape[0]
    if elem_vert.shape != (n_elem, 8) or restriction.shape != (n_elem, (p + 1) ** 3) or vert_xyz.shape[1] != 3:
        raise ValueError("shape mismatch in hx_mesh_create arguments")
    dptr = None
    if dirichlet is not None:
        dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        if dirichlet.size != n_dof:
            raise ValueError("dirichlet must have n_dof entries")
        dptr = ctypes.c_void_p(dirichlet.ctypes.data)
    out = ctypes.c_void_p()
    _check(_lib.hx_mesh_create(p, q, vert_xyz.shape[0], ctypes.c_void_p(vert_xyz.ctypes.data), n_elem,
                               ctypes.c_void_p(elem_vert.ctypes.data), int(n_dof),
                               ctypes.c_void_p(restriction.ctypes.data), dptr, ctypes.byref(out)))
    return out


def hx_mesh_create_structured(nx, ny, nz, p, q, vert_xyz):
    vert_xyz = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    if nx < 1 or ny < 1 or nz < 1:
        # still handed to the library, which reports HX_ERR_ARG
        return _check_none(_lib.hx_mesh_create_structured(nx, ny, nz, p, q, ctypes.c_void_p(vert_xyz.ctypes.data),
                                                          ctypes.byref(ctypes.c_void_p())))
    if vert_xyz.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
        raise ValueError("vert_xyz must be ((nx+1)(ny+1)(nz+1), 3)")
    out = ctypes.c_void_p()
    _check(_lib.hx_mesh_create_structured(nx, ny, nz, p, q, ctypes.c_void_p(vert_xyz.ctypes.data), ctypes.byref(out)))
    return out


def hx_mesh_create_box(nx, ny, nz, p, q, vert_xyz, dirichlet_faces=63):
    vert_xyz = np.ascontiguousarray(vert_xyz, dtype=np.float64)
    if vert_xyz.shape != ((nx + 1) * (ny + 1) * (nz + 1), 3):
        raise ValueError("vert_xyz must be ((nx+1)(ny+1)(nz+1), 3)")
    out = ctypes.c_void_p()
    _check(_lib.hx_mesh_create_box(nx, ny, nz, p, q, ctypes.c_void_p(vert_xyz.ctypes.data), int(dirichlet_faces),
                                   ctypes.byref(out)))
    return out


def _check_none(status):
    _check(status)
    return None


def hx_mesh_destroy(mesh):
    _lib.hx_mesh_destroy(mesh)


def _info(fn, h):
    E, n, p, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    _check(fn(h, ctypes.byref(E), ctypes.byref(n), ctypes.byref(p), ctypes.byref(q)))
    return E.value, n.value, p.value, q.value


def hx_mesh_info(mesh):
    return _info(_lib.hx_mesh_info, mesh)


def hx_op_info(op):
    return _info(_lib.hx_op_info, op)


def hx_mesh_qpoint_coords(mesh, xyz, stream=None):
    E, _, _, q = hx_mesh_info(mesh)
    _check(_lib.hx_mesh_qpoint_coords(mesh, _dptr(xyz, E * q ** 3 * 3, "xyz"), _stream(stream)))


def hx_mesh_node_coords(mesh, xyz, stream=None):
    _, n, _, _ = hx_mesh_info(mesh)
    _check(_lib.hx_mesh_node_coords(mesh, _dptr(xyz, n * 3, "xyz"), _stream(stream)))


def hx_op_create(mesh, alpha, nu, nu_q=None, geom_mode=HX_GEOM_STORED, stream=None):
    E, _, _, q = hx_mesh_info(mesh)
    nptr = None if nu_q is None else _dptr(nu_q, E * q ** 3, "nu_q")
    out = ctypes.c_void_p()
    _check(_lib.hx_op_create(mesh, float(alpha), float(nu), nptr, int(geom_mode), _stream(stream), ctypes.byref(out)))
    return out


def hx_op_set_coefficients(op, alpha, nu, nu_q=None, stream=None):
    E, _, _, q = hx_op_info(op)
    nptr = None if nu_q is None else _dptr(nu_q, E * q ** 3, "nu_q")
    _check(_lib.hx_op_set_coefficients(op, float(alpha), float(nu), nptr, _stream(stream)))


def hx_op_launch_count(op) -> int:
    return int(_lib.hx_op_launch_count(op))


def hx_op_destroy(op):
    _lib.hx_op_destroy(op)


def hx_op_apply(op, x, y, constrained=False, stream=None):
    n = hx_op_info(op)[1]
    _check(_lib.hx_op_apply(op, _dptr(x, n, "x"), _dptr(y, n, "y"), int(bool(constrained)), _stream(stream)))


def hx_op_diagonal(op, diag, constrained=False, stream=None):
    n = hx_op_info(op)[1]
    _check(_lib.hx_op_diagonal(op, _dptr(diag, n, "diag"), int(bool(constrained)), _stream(stream)))


def hx_op_load_vector(op, f_q, b, stream=None):
    E, n, _, q = hx_op_info(op)
    _check(_lib.hx_op_load_vector(op, _dptr(f_q, E * q ** 3, "f_q"), _dptr(b, n, "b"), _stream(stream)))


def hx_solve_pcg(op, b, x, rtol=1e-10, max_it=10000, use_x0=False, stream=None, raise_on_fail=True):
    n = hx_op_info(op)[1]
    info = SolveInfo()
    st = _lib.hx_solve_pcg(op, _dptr(b, n, "b"), _dptr(x, n, "x"), float(rtol), int(max_it), int(bool(use_x0)),
                           _stream(stream), ctypes.byref(info))
    if raise_on_fail or st not in (HX_OK, HX_ERR_NOT_CONVERGED, HX_ERR_BREAKDOWN):
        _check(st)
    return info.as_dict()


def hx_solve_pcg_host(op, b_host, x_host, rtol=1e-10, max_it=10000, use_x0=False, stream=None, raise_on_fail=True):
    n = hx_op_info(op)[1]
    info = SolveInfo()
    st = _lib.hx_solve_pcg_host(op, _hptr(b_host, n, "b_host"), _hptr(x_host, n, "x_host"), float(rtol),
                                int(max_it), int(bool(use_x0)), _stream(stream), ctypes.byref(info))
    if raise_on_fail or st not in (HX_OK, HX_ERR_NOT_CONVERGED, HX_ERR_BREAKDOWN):
        _check(st)
    return info.as_dict()


def _fptr(t, n, name):
    """Device pointer of a contiguous float32 CUDA tensor with n elements."""
    if not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.float32" or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def hx_solve_pcg_mixed(op, b, x, rtol=1e-10, max_it=100000, inner_rtol=1e-5, stream=None, raise_on_fail=True):
    n = hx_op_info(op)[1]
    info = SolveInfo()
    st = _lib.hx_solve_pcg_mixed(op, _dptr(b, n, "b"), _dptr(x, n, "x"), float(rtol), int(max_it), float(inner_rtol),
                                 _stream(stream), ctypes.byref(info))
    if raise_on_fail or st not in (HX_OK, HX_ERR_NOT_CONVERGED, HX_ERR_BREAKDOWN):
        _check(st)
    return info.as_dict()


def hx_op_apply_f32(op, x, y, stream=None):
    n = hx_op_info(op)[1]
    _check(_lib.hx_op_apply_f32(op, _fptr(x, n, "x"), _fptr(y, n, "y"), _stream(stream)))


def hx_probe_fma(fp64, iters, stream=None):
    """Enqueue the FMA-throughput probe; returns the flops the launch performs."""
    f = _D(0.0)
    _check(_lib.hx_probe_fma(1 if fp64 else 0, int(iters), _stream(stream), ctypes.byref(f)))
    return f.value


HX_F32_AUTO, HX_F32_COLLOCATED, HX_F32_DIRECT_STAGED, HX_F32_DIRECT = -1, 0, 1, 2
HX_F32_MMA_BF16, HX_F32_MMA_BF16X3 = 3, 4


def hx_op_set_f32_kernel(op, kind):
    _check(_lib.hx_op_set_f32_kernel(op, int(kind)))


def hx_op_set_f32_tile(op, tile):
    _check(_lib.hx_op_set_f32_tile(op, int(tile)))


def hx_op_f32_kernel(op):
    """(kind in use or -1, elements per block or -1, [autotuner ms per launch of each kind's fastest
    tile, -1 where not timed])"""
    k, ne = _I(0), _I(0)
    ms = (ctypes.c_float * 3)()
    _check(_lib.hx_op_f32_kernel(op, ctypes.byref(k), ctypes.byref(ne), ms))
    return k.value, ne.value, list(ms)


def hx_op_set_wait_limit(op, attempts):
    _check(_lib.hx_op_set_wait_limit(op, int(attempts)))


def hx_op_gradient(op, u, lam, dnu_q, df_q, stream=None):
    E, n, _, q = hx_op_info(op)
    _check(_lib.hx_op_gradient(op, _dptr(u, n, "u"), _dptr(lam, n, "lam"), _dptr(dnu_q, E * q ** 3, "dnu_q"),
                               _dptr(df_q, E * q ** 3, "df_q"), _stream(stream)))


def hx_op_collocated_mass(op, diag, stream=None):
    n = hx_op_info(op)[1]
    _check(_lib.hx_op_collocated_mass(op, _dptr(diag, n, "diag"), _stream(stream)))


def hx_op_set_preconditioner(op, kind, degree=8, stream=None):
    _check(_lib.hx_op_set_preconditioner(op, int(kind), int(degree), _stream(stream)))


def hx_op_lor_csr(op, row_off=None, col=None, val=None, stream=None):
    """Number of stored entries of A_LOR; copies the CSR arrays into the given device tensors."""
    nnz = ctypes.c_int64(0)
    _check(_lib.hx_op_lor_csr(op, ctypes.byref(nnz), None, None, None, _stream(stream)))
    n = hx_op_info(op)[1]
    k = nnz.value
    if row_off is not None or col is not None or val is not None:
        _check(_lib.hx_op_lor_csr(op, ctypes.byref(nnz), _lptr(row_off, n + 1, "row_off") if row_off is not None else None,
                                  _iptr(col, k, "col") if col is not None else None,
                                  _dptr(val, k, "val") if val is not None else None, _stream(stream)))
    return k


def hx_op_precond_apply(op, r, z, stream=None):
    n = hx_op_info(op)[1]
    _check(_lib.hx_op_precond_apply(op, _dptr(r, n, "r"), _dptr(z, n, "z"), _stream(stream)))


def hx_batch_create(ops, b, x, rtol=1e-10, max_it=10000, lanes=0):
    """ops: operator handles; b, x: CUDA float64 tensors (n_dof_i each), bound to the batch;
    lanes: concurrent chains of solves (0: all instances at once; < 0: chosen by timing at the
    first solve)."""
    n = len(ops)
    if not (len(b) == len(x) == n) or n < 1:
        raise ValueError("ops, b and x must have the same positive length")
    H = (ctypes.c_void_p * n)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in ops])
    Bp = (ctypes.c_void_p * n)(*[_dptr(bi, hx_op_info(o)[1], f"b[{i}]").value for i, (o, bi) in enumerate(zip(ops, b))])
    Xp = (ctypes.c_void_p * n)(*[_dptr(xi, hx_op_info(o)[1], f"x[{i}]").value for i, (o, xi) in enumerate(zip(ops, x))])
    out = ctypes.c_void_p()
    _check(_lib.hx_batch_create(n, ctypes.cast(H, ctypes.c_void_p), ctypes.cast(Bp, ctypes.c_void_p),
                                ctypes.cast(Xp, ctypes.c_void_p), float(rtol), int(max_it), int(lanes),
                                ctypes.byref(out)))
    return out


def hx_batch_solve(batch, n, stream=None, raise_on_fail=True):
    infos = (SolveInfo * n)()
    st = _lib.hx_batch_solve(batch, _stream(stream), ctypes.cast(infos, ctypes.c_void_p))
    if raise_on_fail or st not in (HX_OK, HX_ERR_NOT_CONVERGED, HX_ERR_BREAKDOWN):
        _check(st)
    return [i.as_dict() for i in infos]


def hx_batch_lanes(batch):
    return _lib.hx_batch_lanes(batch)


def hx_batch_destroy(batch):
    _lib.hx_batch_destroy(batch)


HX_BATCH_AUTO, HX_BATCH_FUSED = -1, -2


class Batch:
    """Owning handle of a batch; keeps its operators and vectors alive.  lanes: chains of solves
    (0: all concurrent), HX_BATCH_FUSED (lock-step iterations), HX_BATCH_AUTO (timed choice)."""

    def __init__(self, ops, b, x, rtol=1e-10, max_it=10000, lanes=0):
        self.ops, self.b, self.x = list(ops), list(b), list(x)
        self.handle = hx_batch_create([o.handle for o in self.ops], self.b, self.x, rtol, max_it, lanes)

    def solve(self, stream=None, raise_on_fail=True):
        return hx_batch_solve(self.handle, len(self.ops), stream, raise_on_fail)

    @property
    def lanes(self):
        """Lanes of the next solve, or HX_BATCH_FUSED (after autotuning: the chosen one)."""
        return hx_batch_lanes(self.handle)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h is not None and _lib is not None:
            _lib.hx_batch_destroy(h)


def _lptr(t, n, name):
    """Device pointer of a contiguous int64 CUDA tensor with n elements."""
    if not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.int64" or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int64 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _iptr(t, n, name):
    """Device pointer of a contiguous int32 CUDA tensor with n elements."""
    if not getattr(t, "is_cuda", False) or str(t.dtype) != "torch.int32" or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def hx_apply_noalloc(p, q, X8, restriction, t_offsets, t_indices, alpha, nu, x, y, stream=None):
    """y = A x without any device allocation (see include/hx.h): every array comes from the caller."""
    n_elem = int(restriction.shape[0])
    n_dof = int(x.numel())
    n3 = (p + 1) ** 3
    _check(_lib.hx_apply_noalloc(int(p), int(q), n_elem, n_dof, _dptr(X8, n_elem * 24, "X8"),
                                 _iptr(restriction, n_elem * n3, "restriction"), _iptr(t_offsets, n_dof + 1, "t_offsets"),
                                 _iptr(t_indices, n_elem * n3, "t_indices"), float(alpha), float(nu),
                                 _dptr(x, n_dof, "x"), _dptr(y, n_dof, "y"), _stream(stream)))


# ---------------------------------------------------------------------------
# owning handles (destroyed on garbage collection); still marshalling only
# ---------------------------------------------------------------------------
class Mesh:
    def __init__(self, handle):
        self.handle = handle
        self.n_elem, self.n_dof, self.p, self.q = hx_mesh_info(handle)

    @classmethod
    def structured(cls, nx, ny, nz, p, q, vert_xyz):
        return cls(hx_mesh_create_structured(nx, ny, nz, p, q, vert_xyz))

    @classmethod
    def box(cls, nx, ny, nz, p, q, vert_xyz, dirichlet_faces=63):
        return cls(hx_mesh_create_box(nx, ny, nz, p, q, vert_xyz, dirichlet_faces))

    @classmethod
    def general(cls, p, q, vert_xyz, elem_vert, n_dof, restriction, dirichlet=None):
        return cls(hx_mesh_create(p, q, vert_xyz, elem_vert, n_dof, restriction, dirichlet))

    def qpoint_coords(self, stream=None):
        import torch
        out = torch.empty((self.n_elem, self.q ** 3, 3), dtype=torch.float64, device="cuda")
        hx_mesh_qpoint_coords(self.handle, out, stream)
        return out

    def node_coords(self, stream=None):
        import torch
        out = torch.empty((self.n_dof, 3), dtype=torch.float64, device="cuda")
        hx_mesh_node_coords(self.handle, out, stream)
        return out

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h is not None and _lib is not None:
            _lib.hx_mesh_destroy(h)


class Operator:
    def __init__(self, mesh: Mesh, alpha, nu, nu_q=None, geom_mode=HX_GEOM_STORED, stream=None):
        self.mesh = mesh  # keeps the mesh alive
        self.handle = hx_op_create(mesh.handle, alpha, nu, nu_q, geom_mode, stream)
        self.n_dof = mesh.n_dof
        self.coef_token = object()

    def apply(self, x, y=None, constrained=False, stream=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        hx_op_apply(self.handle, x, y, constrained, stream)
        return y

    def diagonal(self, constrained=False, stream=None):
        import torch
        d = torch.empty(self.n_dof, dtype=torch.float64, device="cuda")
        hx_op_diagonal(self.handle, d, constrained, stream)
        return d

    def load_vector(self, f_q, stream=None):
        import torch
        b = torch.empty(self.n_dof, dtype=torch.float64, device="cuda")
        hx_op_load_vector(self.handle, f_q, b, stream)
        return b

    def set_coefficients(self, alpha, nu, nu_q=None, stream=None):
        hx_op_set_coefficients(self.handle, alpha, nu, nu_q, stream)
        self.coef_token = object()  # identifies the coefficients now set

    def launch_count(self):
        return hx_op_launch_count(self.handle)

    def solve(self, b, x=None, rtol=1e-10, max_it=10000, stream=None, raise_on_fail=True):
        import torch
        use_x0 = x is not None
        x = torch.zeros_like(b) if x is None else x
        info = hx_solve_pcg(self.handle, b, x, rtol, max_it, use_x0, stream, raise_on_fail)
        return x, info

    def solve_mixed(self, b, rtol=1e-10, inner_rtol=1e-5, max_it=100000, stream=None, raise_on_fail=True):
        import torch
        x = torch.empty_like(b)
        info = hx_solve_pcg_mixed(self.handle, b, x, rtol, max_it, inner_rtol, stream, raise_on_fail)
        return x, info

    def collocated_mass(self, stream=None):
        """alpha Mc, the Gauss-Lobatto collocated (diagonal) mass, as an n_dof vector."""
        import torch
        d = torch.empty(self.n_dof, dtype=torch.float64, device="cuda")
        hx_op_collocated_mass(self.handle, d, stream)
        return d

    def set_preconditioner(self, kind, degree=8, stream=None):
        hx_op_set_preconditioner(self.handle, kind, degree, stream)

    def lor_csr(self, stream=None):
        """(row_off, col, val) of the assembled low-order refined matrix (Sec. 5.2), device tensors."""
        import torch
        k = hx_op_lor_csr(self.handle, stream=stream)
        row_off = torch.empty(self.n_dof + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(k, dtype=torch.int32, device="cuda")
        val = torch.empty(k, dtype=torch.float64, device="cuda")
        hx_op_lor_csr(self.handle, row_off, col, val, stream)
        return row_off, col, val

    def precond_apply(self, r, stream=None):
        import torch
        z = torch.empty_like(r)
        hx_op_precond_apply(self.handle, r, z, stream)
        return z

    def gradient(self, u, lam, stream=None):
        """(dL/dnu_q, dL/df_q), each n_elem x q^3, from the solution u and the adjoint lam."""
        import torch
        shape = (self.mesh.n_elem, self.mesh.q ** 3)
        dnu = torch.empty(shape, dtype=torch.float64, device="cuda")
        df = torch.empty(shape, dtype=torch.float64, device="cuda")
        hx_op_gradient(self.handle, u, lam, dnu, df, stream)
        return dnu, df

    def apply_f32(self, x, stream=None):
        import torch
        y = torch.empty_like(x)
        hx_op_apply_f32(self.handle, x, y, stream)
        return y

    def set_wait_limit(self, attempts):
        hx_op_set_wait_limit(self.handle, attempts)

    def set_f32_kernel(self, kind):
        hx_op_set_f32_kernel(self.handle, kind)

    def set_f32_tile(self, tile):
        hx_op_set_f32_tile(self.handle, tile)

    def f32_kernel(self):
        return hx_op_f32_kernel(self.handle)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h is not None and _lib is not None:
            _lib.hx_op_destroy(h)


__all__ = list(SIGNATURES) + ["Mesh", "Operator", "Batch", "HxError", "SolveInfo", "LIB_PATH", "HX_GEOM_STORED",
                              "HX_GEOM_ONTHEFLY", "HX_PREC_JACOBI", "HX_PREC_COLLOCATED_MASS",
                              "HX_PREC_LOR", "HX_PREC_LOR_MC", "HX_PREC_LOR_MG", "HX_F32_AUTO", "HX_F32_COLLOCATED",
                              "HX_F32_DIRECT_STAGED", "HX_F32_DIRECT", "HX_F32_MMA_BF16", "HX_F32_MMA_BF16X3",
                              "HX_BATCH_AUTO", "HX_BATCH_FUSED"]
