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
* ``direct3d`` / ``fmm3d`` (and ``bin3d``, ``sort3d``, ``interaction_list3d``,
  the operators ``p2m3d`` ... ``l2p3d``) -- the three-dimensional extension
                      the paper names first (Sec. 8): the Laplace potential
                      and field of point charges, directly and by the FMM on
                      a uniform octree with solid-harmonic series
                      (``oracle3d.c``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC3 = os.path.join(_HERE, "oracle3d.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EDOMAIN = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O2, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC3))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, _SRC3, "-o", tmp, "-lm"]
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
        # three dimensions (oracle3d.c)
        lib.o3_harmonics.argtypes = [f64, f64, f64, i32, P, P]
        lib.o3_harmonics.restype = i32
        lib.o3_direct.argtypes = [i64, P, P, P, P, i64, P, P, P, P, P]
        lib.o3_direct.restype = i32
        lib.o3_morton.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, i32]
        lib.o3_morton.restype = ctypes.c_uint32
        lib.o3_bin.argtypes = [i64, P, P, P, f64, f64, f64, f64, i32, P]
        lib.o3_bin.restype = i32
        lib.o3_sort.argtypes = [i64, P, i32, P, P]
        lib.o3_sort.restype = i32
        lib.o3_interaction_list.argtypes = [i32, i32, i32, i32, P]
        lib.o3_interaction_list.restype = i32
        lib.o3_p2m.argtypes = [i64, P, P, P, P, P, i32, P]
        lib.o3_p2m.restype = None
        for name in ("o3_m2m", "o3_m2l", "o3_l2l"):
            fn = getattr(lib, name)
            fn.argtypes = [i32, P, P, P, P]
            fn.restype = None
        lib.o3_l2p.argtypes = [i32, P, P, f64, f64, f64, P]
        lib.o3_l2p.restype = None
        lib.o3_me_eval.argtypes = [i32, P, P, f64, f64, f64]
        lib.o3_me_eval.restype = f64
        lib.o3_fmm.argtypes = [i64, P, P, P, P, f64, f64, f64, f64, i32, i32, P, P, P, P]
        lib.o3_fmm.restype = i32
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


# ---------------------------------------------------------------------------
# Three dimensions (oracle3d.c): the 3D Laplace potential and field of point
# charges, directly and by the FMM on a uniform octree -- the extension the
# paper names first in its conclusions (Sec. 8), with the solid-harmonic
# series written out in oracle3d.c.  Expansions are arrays of p * (2p - 1)
# complex coefficients, index n (2p - 1) + m + p - 1 for degree n < p and
# order -n <= m <= n (entries with |m| > n unused).
# ---------------------------------------------------------------------------
def idx3(p, n, m):
    """Index of coefficient (n, m) in a 3D expansion of p terms."""
    return n * (2 * p - 1) + m + p - 1


def _cplx(a, size):
    out = np.zeros(size, dtype=np.complex128) if a is None else np.ascontiguousarray(
        a, dtype=np.complex128).copy()
    assert out.size == size
    return out


def harmonics3d(v, P, irregular=True):
    """Regular R_n^m(v) and irregular I_n^m(v) solid harmonics, n < P, as
    (P, 2P - 1) complex arrays indexed [n, m + P - 1]."""
    lib = _load()
    R = np.zeros(P * (2 * P - 1), np.complex128)
    Iv = np.zeros(P * (2 * P - 1), np.complex128) if irregular else None
    _check(lib.o3_harmonics(float(v[0]), float(v[1]), float(v[2]), P, R.ctypes.data,
                            _ptr(Iv)), "harmonics3d")
    return R.reshape(P, 2 * P - 1), (None if Iv is None else Iv.reshape(P, 2 * P - 1))


def direct3d(x, y, z, q, targets=None):
    """D3: potential sum_{j != i} q_j / r_ij and field -grad of it at each
    target (all particles if targets is None)."""
    lib = _load()
    x, y, z, q = _f64(x), _f64(y), _f64(z), _f64(q)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = x.size if t is None else t.size
    phi, ex, ey, ez = (np.zeros(nt) for _ in range(4))
    _check(lib.o3_direct(x.size, x.ctypes.data, y.ctypes.data, z.ctypes.data, q.ctypes.data, nt,
                         _ptr(t), phi.ctypes.data, ex.ctypes.data, ey.ctypes.data,
                         ez.ctypes.data), "direct3d")
    return phi, ex, ey, ez


def morton3d(ix, iy, iz, L):
    return int(_load().o3_morton(ix, iy, iz, L))


def bin3d(x, y, z, domain, L):
    """Morton keys of the leaves (domain = (x0, y0, z0, W))."""
    lib = _load()
    x, y, z = _f64(x), _f64(y), _f64(z)
    key = np.zeros(x.size, np.uint32)
    _check(lib.o3_bin(x.size, x.ctypes.data, y.ctypes.data, z.ctypes.data, float(domain[0]),
                      float(domain[1]), float(domain[2]), float(domain[3]), L, key.ctypes.data),
           "bin3d")
    return key


def sort3d(key, L):
    """(perm, start): stable order by key, and the 8^L + 1 leaf starts."""
    lib = _load()
    key = np.ascontiguousarray(key, dtype=np.uint32)
    perm = np.zeros(key.size, np.uint32)
    start = np.zeros((1 << (3 * L)) + 1, np.uint32)
    _check(lib.o3_sort(key.size, key.ctypes.data, L, perm.ctypes.data, start.ctypes.data),
           "sort3d")
    return perm, start


def interaction_list3d(l, ix, iy, iz):
    """(k, 3) array of the source boxes, ascending Morton order."""
    out = np.zeros(3 * 189, np.int32)
    k = _load().o3_interaction_list(l, ix, iy, iz, out.ctypes.data)
    return out[:3 * k].reshape(k, 3)


def p2m3d(x, y, z, q, c, p):
    lib = _load()
    x, y, z, q = _f64(x), _f64(y), _f64(z), _f64(q)
    M = np.zeros(p * (2 * p - 1), np.complex128)
    lib.o3_p2m(x.size, x.ctypes.data, y.ctypes.data, z.ctypes.data, q.ctypes.data,
               _f64(c).ctypes.data, p, M.ctypes.data)
    return M


def m2m3d(M, c, cp, p):
    """Shift a multipole expansion from centre c to centre cp."""
    out = _cplx(None, p * (2 * p - 1))
    M = _cplx(M, out.size)
    _load().o3_m2m(p, M.ctypes.data, _f64(c).ctypes.data, _f64(cp).ctypes.data, out.ctypes.data)
    return out


def m2l3d(M, cs, ct, p):
    """Local expansion about ct of the multipole expansion M about cs."""
    out = _cplx(None, p * (2 * p - 1))
    M = _cplx(M, out.size)
    _load().o3_m2l(p, M.ctypes.data, _f64(cs).ctypes.data, _f64(ct).ctypes.data, out.ctypes.data)
    return out


def l2l3d(Lc, c, cc, p):
    """Shift a local expansion from centre c to centre cc."""
    out = _cplx(None, p * (2 * p - 1))
    Lc = _cplx(Lc, out.size)
    _load().o3_l2l(p, Lc.ctypes.data, _f64(c).ctypes.data, _f64(cc).ctypes.data, out.ctypes.data)
    return out


def l2p3d(Lc, c, pt, p):
    """(phi, ex, ey, ez) of a local expansion about c at point pt."""
    out = np.zeros(4)
    Lc = _cplx(Lc, p * (2 * p - 1))
    _load().o3_l2p(p, Lc.ctypes.data, _f64(c).ctypes.data, float(pt[0]), float(pt[1]),
                   float(pt[2]), out.ctypes.data)
    return tuple(out)


def me_eval3d(M, c, pt, p):
    """Potential of a multipole expansion about c at point pt."""
    M = _cplx(M, p * (2 * p - 1))
    return float(_load().o3_me_eval(p, M.ctypes.data, _f64(c).ctypes.data, float(pt[0]),
                                    float(pt[1]), float(pt[2])))


def fmm3d(x, y, z, q, domain, L, p):
    """F3: (phi, ex, ey, ez) of every particle by the FMM on the uniform
    octree of depth L (1..6) with p terms; domain = (x0, y0, z0, W)."""
    lib = _load()
    x, y, z, q = _f64(x), _f64(y), _f64(z), _f64(q)
    n = x.size
    phi, ex, ey, ez = (np.zeros(n) for _ in range(4))
    _check(lib.o3_fmm(n, x.ctypes.data, y.ctypes.data, z.ctypes.data, q.ctypes.data,
                      float(domain[0]), float(domain[1]), float(domain[2]), float(domain[3]), L,
                      p, phi.ctypes.data, ex.ctypes.data, ey.ctypes.data, ez.ctypes.data),
           "fmm3d")
    return phi, ex, ey, ez
