"""FP64 CPU oracle for the 2D vortex-blob FMM evaluation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  The product (``paper_0905_2637_gb300``) never imports
it, and it imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no fused multiply-add);
this module compiles it with gcc on first use and wraps it with ctypes.
Every function cites the passage of the PetFMM paper it follows:

* ``direct``       -- O1, Eq. 9 with the regularised kernel of Eq. 8.
* ``substituted``  -- O2, Eq. 9 with the far pairs on the singular kernel of
                      Eq. 7 (kernel substitution, end of Sec. 3).
* ``fmm``          -- O3, the FMM of Sec. 2.2 / Fig. 2 (P2M, M2M, M2L, L2L,
                      L2P, P2P) on the uniform quadtree of Sec. 2.1.
* ``bin`` / ``sort`` / ``interaction_list`` -- the tree of Sec. 2.1 with the
                      z-order numbering of Sec. 5.1 and the interaction list
                      of Sec. 2.2 (at most 27 members, Table 1).
* ``laplace_direct`` / ``laplace_fmm`` -- the second kernel (the Evaluator of
                      Sec. 6.1 takes the kernel as a parameter): the 2D
                      logarithmic potential sum_{j != i} q_j log|x_i - x_j|,
                      directly and by the FMM of Sec. 2.2 with the series of
                      the complex logarithm.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EDOMAIN = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O2, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_direct.argtypes = [i64, P, P, P, f64, i64, P, P, P, i32]
        lib.orc_direct.restype = None
        lib.orc_substituted.argtypes = [i64, P, P, P, f64, f64, f64, i32, f64, i64, P, P, P, i32]
        lib.orc_substituted.restype = i32
        lib.orc_bin.argtypes = [i64, P, P, f64, f64, f64, i32, P, P, P]
        lib.orc_bin.restype = i32
        lib.orc_sort.argtypes = [i64, P, i32, P, P]
        lib.orc_sort.restype = i32
        lib.orc_interaction_list.argtypes = [i32, i32, i32, P]
        lib.orc_interaction_list.restype = i32
        lib.orc_morton.argtypes = [ctypes.c_uint32, ctypes.c_uint32, i32]
        lib.orc_morton.restype = ctypes.c_uint32
        lib.orc_fmm.argtypes = [i64, P, P, P, f64, f64, f64, i32, i32, f64, i64, P, P, P, P, P, i32]
        lib.orc_fmm.restype = i32
        lib.orc_kernel_sigma.argtypes = [f64, f64, f64, P, P]
        lib.orc_kernel_sigma.restype = None
        lib.orc_p2m.argtypes = [i64, P, P, P, f64, f64, i32, P]
        lib.orc_p2m.restype = None
        for name in ("orc_m2m", "orc_m2l", "orc_l2l", "orc_l2p", "orc_me_eval",
                     "orc_lap_m2m", "orc_lap_m2l", "orc_lap_me_eval"):
            fn = getattr(lib, name)
            fn.argtypes = [i32, P, f64, f64, f64, f64, P]
            fn.restype = None
        lib.orc_lap_p2m.argtypes = [i64, P, P, P, f64, f64, i32, P]
        lib.orc_lap_p2m.restype = None
        lib.orc_laplace_direct.argtypes = [i64, P, P, P, i64, P, P, i32]
        lib.orc_laplace_direct.restype = None
        lib.orc_laplace_fmm.argtypes = [i64, P, P, P, f64, f64, f64, i32, i32, i64, P, P, P, P,
                                        i32]
        lib.orc_laplace_fmm.restype = i32
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = i32
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != ORC_OK:
        names = {ORC_EINVAL: "EINVAL", ORC_ENOMEM: "ENOMEM", ORC_EDOMAIN: "EDOMAIN"}
        raise OracleError(rc, f"{what}: {names.get(rc, rc)}")


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


def max_threads() -> int:
    return int(_load().orc_max_threads())


def kernel_sigma(dx: float, dy: float, sigma: float):
    """K_sigma(x) of Eq. 8 for a unit-strength source at offset (dx, dy)."""
    lib = _load()
    ku, kv = ctypes.c_double(), ctypes.c_double()
    lib.orc_kernel_sigma(dx, dy, sigma, ctypes.byref(ku), ctypes.byref(kv))
    return ku.value, kv.value


def direct(x, y, g, sigma, targets=None, nthreads=0):
    """O1 (Eq. 9): velocity of every target from all other particles."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(g)
    n = x.size
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.size
    u, v = np.zeros(nt), np.zeros(nt)
    lib.orc_direct(n, _ptr(x), _ptr(y), _ptr(g), float(sigma), nt, _ptr(t), _ptr(u), _ptr(v), nthreads)
    return u, v


def substituted(x, y, g, domain, L, sigma, targets=None, nthreads=0):
    """O2: near pairs (leaf distance <= 1) on Eq. 8, far pairs on Eq. 7."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(g)
    n = x.size
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.size
    u, v = np.zeros(nt), np.zeros(nt)
    x0, y0, W = domain
    rc = lib.orc_substituted(n, _ptr(x), _ptr(y), _ptr(g), x0, y0, W, L, float(sigma), nt,
                             _ptr(t), _ptr(u), _ptr(v), nthreads)
    _check(rc, "substituted")
    return u, v


def bin(x, y, domain, L):
    """Leaf coordinates (ix, iy) and Morton keys (Sec. 2.1, z-order Sec. 5.1)."""
    lib = _load()
    x, y = _f64(x), _f64(y)
    n = x.size
    ix = np.zeros(n, np.uint32)
    iy = np.zeros(n, np.uint32)
    key = np.zeros(n, np.uint32)
    x0, y0, W = domain
    rc = lib.orc_bin(n, _ptr(x), _ptr(y), x0, y0, W, L, _ptr(ix), _ptr(iy), _ptr(key))
    _check(rc, "bin")
    return ix, iy, key


def sort(key, L):
    """Stable sort by key: (perm, start) with start[b] = first rank of leaf b."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint32)
    perm = np.zeros(key.size, np.uint32)
    start = np.zeros((1 << (2 * L)) + 1, np.uint32)
    rc = lib.orc_sort(key.size, _ptr(key), L, _ptr(perm), _ptr(start))
    _check(rc, "sort")
    return perm, start


def morton(ix, iy, L):
    return int(_load().orc_morton(int(ix), int(iy), int(L)))


def interaction_list(level, ix, iy):
    """Interaction list of box (level, ix, iy) as an (n, 2) array of source
    box coordinates in ascending Morton order (Sec. 2.2, Table 1)."""
    lib = _load()
    out = np.zeros(2 * 27, np.int32)
    cnt = lib.orc_interaction_list(int(level), int(ix), int(iy), _ptr(out))
    return out[: 2 * cnt].reshape(cnt, 2).copy()


def fmm(x, y, g, domain, L, p, sigma, targets=None, export=False, nthreads=0):
    """O3: textbook FMM velocity (Sec. 2.2).  With ``export`` (all targets
    only) also returns the ME and LE arrays, shape (Lambda, p) complex, box
    index = (4^l - 1)/3 + Morton index at level l."""
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(g)
    n = x.size
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.size
    u, v = np.zeros(nt), np.zeros(nt)
    me = le = None
    if export:
        if t is not None:
            raise ValueError("export needs every particle as a target")
        nbox = ((1 << (2 * (L + 1))) - 1) // 3
        me = np.zeros((nbox, p), np.complex128)
        le = np.zeros((nbox, p), np.complex128)
    x0, y0, W = domain
    rc = lib.orc_fmm(n, _ptr(x), _ptr(y), _ptr(g), x0, y0, W, L, p, float(sigma), nt, _ptr(t),
                     _ptr(u), _ptr(v), _ptr(me), _ptr(le), nthreads)
    _check(rc, "fmm")
    if export:
        return u, v, me, le
    return u, v


# --- single expansion operators (unscaled, p terms), for the pins -------------------------

def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def p2m(x, y, g, zc, p):
    lib = _load()
    x, y, g = _f64(x), _f64(y), _f64(g)
    a = np.zeros(p, np.complex128)
    lib.orc_p2m(x.size, _ptr(x), _ptr(y), _ptr(g), zc.real, zc.imag, p, _ptr(a))
    return a


def _op(name, p, arr, z1, z2):
    lib = _load()
    arr = _c(arr)
    out = np.zeros(p, np.complex128)
    getattr(lib, name)(p, _ptr(arr), z1.real, z1.imag, z2.real, z2.imag, _ptr(out))
    return out


def m2m(a, zc, zp):
    return _op("orc_m2m", len(a), a, complex(zc), complex(zp))


def m2l(a, zs, zt):
    return _op("orc_m2l", len(a), a, complex(zs), complex(zt))


def l2l(b, zp, zc):
    return _op("orc_l2l", len(b), b, complex(zp), complex(zc))


def l2p(b, zl, z):
    lib = _load()
    b = _c(b)
    w = np.zeros(2)
    lib.orc_l2p(len(b), _ptr(b), complex(zl).real, complex(zl).imag, complex(z).real,
                complex(z).imag, _ptr(w))
    return complex(w[0], w[1])


def me_eval(a, zc, z):
    lib = _load()
    a = _c(a)
    w = np.zeros(2)
    lib.orc_me_eval(len(a), _ptr(a), complex(zc).real, complex(zc).imag, complex(z).real,
                    complex(z).imag, _ptr(w))
    return complex(w[0], w[1])


# --- second kernel: the 2D logarithmic potential -------------------------------------------

def laplace_direct(x, y, q, targets=None, nthreads=0):
    """L1: phi_i = sum_{j != i} q_j log|x_i - x_j| (coincident pairs excluded)."""
    lib = _load()
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.size
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.size
    phi = np.zeros(nt)
    lib.orc_laplace_direct(n, _ptr(x), _ptr(y), _ptr(q), nt, _ptr(t), _ptr(phi), nthreads)
    return phi


def laplace_fmm(x, y, q, domain, L, p, targets=None, export=False, nthreads=0):
    """L3: the potential by the FMM of Sec. 2.2 with logarithmic series (p
    terms, the log counted as one).  ``export`` as for ``fmm``."""
    lib = _load()
    x, y, q = _f64(x), _f64(y), _f64(q)
    n = x.size
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.size
    phi = np.zeros(nt)
    me = le = None
    if export:
        if t is not None:
            raise ValueError("export needs every particle as a target")
        nbox = ((1 << (2 * (L + 1))) - 1) // 3
        me = np.zeros((nbox, p), np.complex128)
        le = np.zeros((nbox, p), np.complex128)
    x0, y0, W = domain
    rc = lib.orc_laplace_fmm(n, _ptr(x), _ptr(y), _ptr(q), x0, y0, W, L, p, nt, _ptr(t),
                             _ptr(phi), _ptr(me), _ptr(le), nthreads)
    _check(rc, "laplace_fmm")
    if export:
        return phi, me, le
    return phi


def lap_p2m(x, y, q, zc, p):
    lib = _load()
    x, y, q = _f64(x), _f64(y), _f64(q)
    a = np.zeros(p, np.complex128)
    lib.orc_lap_p2m(x.size, _ptr(x), _ptr(y), _ptr(q), complex(zc).real, complex(zc).imag, p,
                    _ptr(a))
    return a


def lap_m2m(a, zc, zp):
    return _op("orc_lap_m2m", len(a), a, complex(zc), complex(zp))


def lap_m2l(a, zs, zt):
    return _op("orc_lap_m2l", len(a), a, complex(zs), complex(zt))


def lap_me_eval(a, zc, z):
    lib = _load()
    a = _c(a)
    w = np.zeros(2)
    lib.orc_lap_me_eval(len(a), _ptr(a), complex(zc).real, complex(zc).imag, complex(z).real,
                        complex(z).imag, _ptr(w))
    return complex(w[0], w[1])
