"""The three-dimensional extension (the first one the paper names, Sec. 8):
the Laplace potential and field of point charges by the FMM on a uniform
octree, ``petfmm3d_*`` of ``libpetfmm.so``.  Argument marshalling only:
every step runs in the library's kernels, and without the library there is
no fallback."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

STAGES3 = ("bin", "sort", "gather", "p2m", "m2m", "m2l", "l2l", "near")
PETFMM3D_OPT_TIMING = 1
PETFMM3D_OPT_M2L_TC = 2
PETFMM3D_MAX_L, PETFMM3D_MAX_P = 8, 16


class Domain3(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("width", ctypes.c_double)]


_SIGS = False


def lib3():
    global _SIGS
    lib = _lib.load()
    if not _SIGS:
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        for name, res, args in (
                ("petfmm3d_create", I, [ctypes.POINTER(Domain3), I, I, I, I, P,
                                        ctypes.POINTER(ctypes.c_void_p)]),
                ("petfmm3d_evaluate", I, [P, I64, P, P, P, P, P, P, P, P]),
                ("petfmm3d_sync", I, [P]),
                ("petfmm3d_set_option", I, [P, I, I64]),
                ("petfmm3d_stage_times", I, [P, P, I]),
                ("petfmm3d_debug_tree", I, [P, I64, P, P, P]),
                ("petfmm3d_launches", ctypes.c_uint64, [P]),
                ("petfmm3d_debug_m2l_operator", I, [I, I, I, I, P, I64]),
                ("petfmm3d_debug_shift_operator", I, [I, I, I, P, I64]),
                ("petfmm3d_destroy", I, [P])):
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _SIGS = True
    return lib


def petfmm3d_create(domain, levels, order, precision, dtype, cuda_stream=None):
    h = ctypes.c_void_p()
    dom = Domain3(*map(float, domain))
    _lib._ck(lib3().petfmm3d_create(ctypes.byref(dom), int(levels), int(order), int(precision),
                                    int(dtype), cuda_stream, ctypes.byref(h)), "petfmm3d_create")
    return h


def m2l_operator(order, dx, dy, dz):
    """The mixed path's real M2L operator for offset (dx, dy, dz), as the
    library builds it on the host (FP64): a[k, r] = d(output r) / d(input k)."""
    nr = order * order
    out = np.zeros(nr * nr, np.float64)
    _lib._ck(lib3().petfmm3d_debug_m2l_operator(order, dx, dy, dz, out.ctypes.data, out.size),
             "petfmm3d_debug_m2l_operator")
    return out.reshape(nr, nr)


PETFMM3D_SHIFT_M2M, PETFMM3D_SHIFT_L2L = 0, 1


def shift_operator(order, kind, octant):
    """The mixed path's real M2M (kind PETFMM3D_SHIFT_M2M: child of the
    octant to its parent) or L2L (PETFMM3D_SHIFT_L2L: parent to the child)
    operator, as the library builds it on the host (FP64):
    a[k, r] = d(output r) / d(input k)."""
    nr = order * order
    out = np.zeros(nr * nr, np.float64)
    _lib._ck(lib3().petfmm3d_debug_shift_operator(order, kind, octant, out.ctypes.data, out.size),
             "petfmm3d_debug_shift_operator")
    return out.reshape(nr, nr)


class Context3D:
    """One 3D FMM configuration on a CUDA stream (``petfmm3d_create``);
    domain = (x0, y0, z0, W)."""

    def __init__(self, domain, levels, order, precision="mixed", dtype="f32", stream=None):
        torch = _lib._torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.precision = {"fp64": _lib.PETFMM_FP64, "mixed": _lib.PETFMM_MIXED}[precision]
        self.dtype_code = {"f64": _lib.PETFMM_F64, "f32": _lib.PETFMM_F32}[dtype]
        self.torch_dtype = torch.float32 if dtype == "f32" else torch.float64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.domain, self.levels, self.order = tuple(domain), levels, order
        self.handle = petfmm3d_create(domain, levels, order, self.precision, self.dtype_code,
                                      ctypes.c_void_p(self.stream.cuda_stream))

    def close(self):
        if self.handle is not None:
            lib3().petfmm3d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def evaluate(self, x, y, z, q, out=None):
        """Enqueue one evaluation; returns (phi, ex, ey, ez).  ``sync()``
        before use."""
        torch = _lib._torch()
        n = x.numel()
        if out is None:
            out = tuple(torch.empty(n, dtype=self.torch_dtype, device=x.device) for _ in range(4))
        ptrs = [_lib._dev_ptr(t, self.torch_dtype, n, nm) for t, nm in
                zip((x, y, z, q) + tuple(out), ("x", "y", "z", "q", "phi", "ex", "ey", "ez"))]
        _lib._ck(lib3().petfmm3d_evaluate(self.handle, n, *ptrs), "petfmm3d_evaluate")
        return out

    def sync(self):
        return _lib._ck(lib3().petfmm3d_sync(self.handle), "petfmm3d_sync")

    def set_option(self, option, value):
        _lib._ck(lib3().petfmm3d_set_option(self.handle, int(option), int(value)),
                 "petfmm3d_set_option")

    def stage_times(self):
        ms = (ctypes.c_float * len(STAGES3))()
        _lib._ck(lib3().petfmm3d_stage_times(self.handle, ctypes.cast(ms, ctypes.c_void_p),
                                             len(STAGES3)), "petfmm3d_stage_times")
        return {s: float(ms[i]) for i, s in enumerate(STAGES3)}

    def launches(self):
        return int(lib3().petfmm3d_launches(self.handle))

    def debug_tree(self, n):
        """(sorted keys, perm, leaf starts) of the last evaluation."""
        skeys = np.zeros(n, np.uint32)
        perm = np.zeros(n, np.uint32)
        start = np.zeros((1 << (3 * self.levels)) + 1, np.uint32)
        _lib._ck(lib3().petfmm3d_debug_tree(self.handle, n, skeys.ctypes.data, perm.ctypes.data,
                                            start.ctypes.data), "petfmm3d_debug_tree")
        return skeys, perm, start
