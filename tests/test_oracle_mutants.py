"""The oracle's pins catch plausible mistakes: each mutant below is a copy of
oracle.c with one planted error (a wrong sign, index, direction, operand or
dropped term), compiled on the CPU; at least one pin of the battery must fail
for every mutant, and the unmutated source must pass all of them.  CPU only."""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import integrate

from paper_0905_2637_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

MUTANTS = {
    "m2l_sign": ("double sign = (k % 2 == 0) ? -1.0 : 1.0;", "double sign = (k % 2 == 0) ? 1.0 : -1.0;"),
    "m2l_power": ("a[k] * ipow[k + m + 1];", "a[k] * ipow[k + m];"),
    "m2m_transposed_power": ("s += binom(l, k) * a[k] * dpow[l - k];", "s += binom(l, k) * a[k] * dpow[k];"),
    "m2m_direction": ("static void m2m(int p, const cplx *a, cplx zc, cplx zp, cplx *out) {\n    cplx d = zc - zp;",
                      "static void m2m(int p, const cplx *a, cplx zc, cplx zp, cplx *out) {\n    cplx d = zp - zc;"),
    "l2l_direction": ("static void l2l(int p, const cplx *b, cplx zp, cplx zc, cplx *out) {\n    cplx d = zc - zp;",
                      "static void l2l(int p, const cplx *b, cplx zp, cplx zc, cplx *out) {\n    cplx d = zp - zc;"),
    "p2m_power_off_by_one": ("            a[k] += pw;\n            pw *= d;", "            pw *= d;\n            a[k] += pw;"),
    "il_keeps_neighbours": ("if (abs(sx - ix) <= 1 && abs(sy - iy) <= 1) continue;",
                            "if (abs(sx - ix) <= 0 && abs(sy - iy) <= 0) continue;"),
    "l2l_missing_level": ("                m2l(p, me + (level_offset(l) + sm) * p, zs, zt, tmp);\n                for (int k = 0; k < p; ++k) dst[k] += tmp[k];\n            }\n            if (l >= 3) {",
                          "                m2l(p, me + (level_offset(l) + sm) * p, zs, zt, tmp);\n                for (int k = 0; k < p; ++k) dst[k] += tmp[k];\n            }\n            if (l >= 4) {"),
    "l2p_re_im_swapped": ("double su = cimag(w) / (2.0 * ORC_PI);\n            double sv = creal(w) / (2.0 * ORC_PI);",
                          "double su = creal(w) / (2.0 * ORC_PI);\n            double sv = cimag(w) / (2.0 * ORC_PI);"),
    "near_column_dropped": ("            double nu = 0.0, nv = 0.0;\n            for (int dy = -1; dy <= 1; ++dy) {\n                for (int dx = -1; dx <= 1; ++dx) {",
                            "            double nu = 0.0, nv = 0.0;\n            for (int dy = -1; dy <= 1; ++dy) {\n                for (int dx = -1; dx <= 0; ++dx) {"),
    "kernel_width": ("-expm1(-r2 / (2.0 * sigma * sigma))", "-expm1(-r2 / (sigma * sigma))"),
    "kernel_sign": ("    *ku = -dy * f;\n    *kv = dx * f;\n}\n\n/* Singular", "    *ku = dy * f;\n    *kv = -dx * f;\n}\n\n/* Singular"),
    "binning_ceil": ("    double f = floor(s);", "    double f = ceil(s) - 1.0;"),
}


def _compile(src_text, tag):
    d = tempfile.mkdtemp(prefix=f"orc_{tag}_")
    c = os.path.join(d, "o.c")
    so = os.path.join(d, "o.so")
    open(c, "w").write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", c, "-o", so, "-lm"],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_direct.argtypes = [I64, P, P, P, D, I64, P, P, P, I]
    lib.orc_substituted.argtypes = [I64, P, P, P, D, D, D, I, D, I64, P, P, P, I]
    lib.orc_fmm.argtypes = [I64, P, P, P, D, D, D, I, I, D, I64, P, P, P, P, P, I]
    lib.orc_fmm.restype = I
    lib.orc_kernel_sigma.argtypes = [D, D, D, P, P]
    lib.orc_bin.argtypes = [I64, P, P, D, D, D, I, P, P, P]
    lib.orc_bin.restype = I
    return lib


def _arr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _fmm(lib, w, L, p):
    x, y, g = _arr(w.x), _arr(w.y), _arr(w.gamma)
    u, v = np.zeros(w.n), np.zeros(w.n)
    rc = lib.orc_fmm(w.n, x.ctypes.data, y.ctypes.data, g.ctypes.data, 0.0, 0.0, 1.0, L, p, w.sigma,
                     w.n, None, u.ctypes.data, v.ctypes.data, None, None, 1)
    assert rc == 0
    return u, v


def _direct(lib, w):
    x, y, g = _arr(w.x), _arr(w.y), _arr(w.gamma)
    u, v = np.zeros(w.n), np.zeros(w.n)
    lib.orc_direct(w.n, x.ctypes.data, y.ctypes.data, g.ctypes.data, w.sigma, w.n, None,
                   u.ctypes.data, v.ctypes.data, 1)
    return u, v


def _subst(lib, w, L):
    x, y, g = _arr(w.x), _arr(w.y), _arr(w.gamma)
    u, v = np.zeros(w.n), np.zeros(w.n)
    lib.orc_substituted(w.n, x.ctypes.data, y.ctypes.data, g.ctypes.data, 0.0, 0.0, 1.0, L, w.sigma,
                        w.n, None, u.ctypes.data, v.ctypes.data, 1)
    return u, v


def _rel(u, v, ur, vr):
    return float(np.sqrt(np.sum((u - ur) ** 2 + (v - vr) ** 2) / np.sum(ur ** 2 + vr ** 2)))


def _battery(lib):
    """Names of the pins that fail."""
    failed = []
    # Stokes circulation of the Gaussian blob (Eq. 5) vs the kernel (Eq. 8)
    sigma, r = 0.02, 0.03
    circ, _ = integrate.quad(lambda s: math.exp(-s * s / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2) * 2 * math.pi * s,
                             0.0, r, epsabs=0, epsrel=1e-12)
    ku, kv = ctypes.c_double(), ctypes.c_double()
    lib.orc_kernel_sigma(r, 0.0, sigma, ctypes.byref(ku), ctypes.byref(kv))
    if abs(kv.value - circ / (2 * math.pi * r)) > 1e-10 * abs(kv.value):
        failed.append("stokes")
    # binning at box boundaries (x = 1/8, y = 1/4 at L = 3 -> box (1, 2))
    bx, by = _arr([0.125, 1.0]), _arr([0.25, 1.0])
    ix, iy, key = (np.zeros(2, np.uint32) for _ in range(3))
    lib.orc_bin(2, bx.ctypes.data, by.ctypes.data, 0.0, 0.0, 1.0, 3, ix.ctypes.data, iy.ctypes.data,
                key.ctypes.data)
    if list(ix) != [1, 7] or list(iy) != [2, 7]:
        failed.append("binning")
    # L = 1: the FMM is the direct sum
    w1 = W.tiny(400, 3, L=1, p=5, sigma=0.05)
    if _rel(*_fmm(lib, w1, 1, 5), *_direct(lib, w1)) > 1e-13:
        failed.append("level1")
    # FMM -> substituted sum at high order, on a clumped case
    for L in (3, 4):
        w = W.tiny(900, 20 + L, L=L, clustered_frac=0.3)
        us, vs = _subst(lib, w, L)
        if _rel(*_fmm(lib, w, L, 30), us, vs) > 1e-9:
            failed.append(f"converge_L{L}")
    return failed


def test_unmutated_oracle_passes_battery():
    lib = _compile(open(SRC).read(), "orig")
    assert _battery(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_mutant_is_caught(name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    lib = _compile(src.replace(old, new), name)
    assert _battery(lib), f"mutant {name} passes every pin"
