"""Pins of the oracle's second kernel, the 2D logarithmic potential
phi_i = sum_{j != i} q_j log|x_i - x_j| (the Evaluator of Sec. 6.1 takes the
kernel as a parameter; the FMM is that of Sec. 2.2 with the series of the
complex logarithm).  Each pin is fixed by mathematics outside the oracle:

* a ring of N equal charges q at radius R about c: prod_k (z - c - R w^k) =
  (z - c)^N - R^N, so sum_k q log|z - c - R w^k| = q log|(z - c)^N - R^N|
  exactly, and the multipole coefficients about c are a_0 = qN,
  a_{Nm} = -q R^{Nm} / m, all others 0;
* scaling: phi_i(s x) = phi_i(x) + (sum_{j != i} q_j) log s;
* the gradient of phi is sum_j q_j (x_i - x_j) / |x_i - x_j|^2, which is
  2 pi (v, -u) of the singular point-vortex velocity with gamma = q (the
  vortex direct sum, pinned separately);
* the FMM converges to the direct sum geometrically in p.

A battery of planted mistakes (compiled copies of oracle.c) checks that each
fails at least one pin.  CPU only."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")


def ring(n, R, q, c=0j, theta0=0.0):
    z = c + R * np.exp(1j * (theta0 + 2 * np.pi * np.arange(n) / n))
    return z.real.copy(), z.imag.copy(), np.full(n, float(q))


# --- the pins, written against an oracle-like object ------------------------------------

class Api:
    """Calls the Laplace functions of a compiled oracle (the package or a mutant)."""

    def __init__(self, lib):
        self.lib = lib

    def direct(self, x, y, q, targets=None):
        x, y, q = (np.ascontiguousarray(a, np.float64) for a in (x, y, q))
        t = None if targets is None else np.ascontiguousarray(targets, np.int64)
        nt = x.size if t is None else t.size
        phi = np.zeros(nt)
        self.lib.orc_laplace_direct(x.size, x.ctypes.data, y.ctypes.data, q.ctypes.data, nt,
                                    None if t is None else t.ctypes.data, phi.ctypes.data, 1)
        return phi

    def fmm(self, x, y, q, domain, L, p):
        x, y, q = (np.ascontiguousarray(a, np.float64) for a in (x, y, q))
        phi = np.zeros(x.size)
        rc = self.lib.orc_laplace_fmm(x.size, x.ctypes.data, y.ctypes.data, q.ctypes.data,
                                      *domain, L, p, x.size, None, phi.ctypes.data, None, None, 1)
        assert rc == 0
        return phi

    def p2m(self, x, y, q, zc, p):
        x, y, q = (np.ascontiguousarray(a, np.float64) for a in (x, y, q))
        a = np.zeros(p, np.complex128)
        self.lib.orc_lap_p2m(x.size, x.ctypes.data, y.ctypes.data, q.ctypes.data, zc.real,
                             zc.imag, p, a.ctypes.data)
        return a

    def _op(self, name, a, z1, z2):
        a = np.ascontiguousarray(a, np.complex128)
        out = np.zeros(a.size, np.complex128)
        getattr(self.lib, name)(a.size, a.ctypes.data, z1.real, z1.imag, z2.real, z2.imag,
                                out.ctypes.data)
        return out

    def m2m(self, a, zc, zp):
        return self._op("orc_lap_m2m", a, complex(zc), complex(zp))

    def m2l(self, a, zs, zt):
        return self._op("orc_lap_m2l", a, complex(zs), complex(zt))

    def me_eval(self, a, zc, z):
        w = np.zeros(2)
        a = np.ascontiguousarray(a, np.complex128)
        self.lib.orc_lap_me_eval(a.size, a.ctypes.data, zc.real, zc.imag, z.real, z.imag,
                                 w.ctypes.data)
        return w[0]

    def l2p(self, b, zl, z):
        w = np.zeros(2)
        b = np.ascontiguousarray(b, np.complex128)
        self.lib.orc_l2p(b.size, b.ctypes.data, zl.real, zl.imag, z.real, z.imag, w.ctypes.data)
        return w[0]


def _bind(lib):
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_laplace_direct.argtypes = [I64, P, P, P, I64, P, P, I]
    lib.orc_laplace_direct.restype = None
    lib.orc_laplace_fmm.argtypes = [I64, P, P, P, D, D, D, I, I, I64, P, P, P, P, I]
    lib.orc_laplace_fmm.restype = I
    lib.orc_lap_p2m.argtypes = [I64, P, P, P, D, D, I, P]
    lib.orc_lap_p2m.restype = None
    for name in ("orc_lap_m2m", "orc_lap_m2l", "orc_lap_me_eval", "orc_l2p"):
        getattr(lib, name).argtypes = [I, P, D, D, D, D, P]
        getattr(lib, name).restype = None
    lib.orc_direct.argtypes = [I64, P, P, P, D, I64, P, P, P, I]
    lib.orc_direct.restype = None
    return lib


def pin_ring_direct(api):
    # targets of zero charge inside, on no charge, and outside the ring
    n, R, q, c = 24, 0.3, 0.7, 0.5 + 0.45j
    x, y, g = ring(n, R, q, c, theta0=0.2)
    probe = np.array([0.52 + 0.41j, 0.5 + 0.45j, 0.1 + 0.9j, 0.95 + 0.05j])
    xs = np.concatenate([x, probe.real])
    ys = np.concatenate([y, probe.imag])
    qs = np.concatenate([g, np.zeros(probe.size)])
    phi = api.direct(xs, ys, qs, targets=np.arange(n, n + probe.size))
    zz = probe - c
    exact = q * np.log(np.abs(zz ** n - (R ** n) * np.exp(1j * n * 0.2)))
    return np.max(np.abs(phi - exact)) < 1e-12


def pin_scaling(api):
    rng = np.random.default_rng(3)
    x, y, q = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50), rng.uniform(-1, 1, 50)
    s = 2.5
    a, b = api.direct(x, y, q), api.direct(s * x, s * y, q)
    return np.max(np.abs(b - a - (q.sum() - q) * np.log(s))) < 1e-12


def pin_gradient_vs_vortex(api):
    rng = np.random.default_rng(4)
    n = 40
    x, y, q = rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1, 1, n)
    u = np.zeros(n)
    v = np.zeros(n)
    api.lib.orc_direct(n, x.ctypes.data, y.ctypes.data, q.ctypes.data, 1e-12, n, None,
                       u.ctypes.data, v.ctypes.data, 1)
    h = 1e-6
    ok = True
    for i in (0, 7, 23):
        gx = []
        for dxy in ((h, 0.0), (-h, 0.0), (0.0, h), (0.0, -h)):
            xx, yy = x.copy(), y.copy()
            xx[i] += dxy[0]
            yy[i] += dxy[1]
            gx.append(api.direct(xx, yy, q, targets=[i])[0])
        dphx, dphy = (gx[0] - gx[1]) / (2 * h), (gx[2] - gx[3]) / (2 * h)
        # singular vortex velocity: (u, v) = sum g (-dy, dx) / (2 pi r^2)
        ok &= abs(dphx - 2 * np.pi * v[i]) < 1e-6 * (1 + abs(dphx))
        ok &= abs(dphy + 2 * np.pi * u[i]) < 1e-6 * (1 + abs(dphy))
    return bool(ok)


def pin_ring_multipole(api):
    n, R, q, c = 6, 0.1, 1.3, 0.25 + 0.75j
    x, y, g = ring(n, R, q, c)
    p = 20
    a = api.p2m(x, y, g, c, p)
    want = np.zeros(p, np.complex128)
    want[0] = q * n
    for m in range(1, p):
        if (n * m) < p:
            want[n * m] = -q * R ** (n * m) / m
    return np.max(np.abs(a - want)) < 1e-14


def pin_ring_m2m_m2l(api):
    # a ring about c1 translated to c2 (M2M), then to a well-separated local
    # centre zt (M2L), evaluated near zt (L2P): the exact ring potential there,
    # within the geometric truncation error
    n, R, q, c1 = 5, 0.05, 0.9, 0.1 + 0.1j
    x, y, g = ring(n, R, q, c1, theta0=0.3)
    ok = True
    errs = []
    for p in (10, 20, 30):
        a = api.p2m(x, y, g, c1, p)
        c2 = 0.125 + 0.125j
        a2 = api.m2m(a, c1, c2)
        z = 0.9 + 0.6j
        exact = q * np.log(np.abs((z - c1) ** n - (R ** n) * np.exp(1j * n * 0.3)))
        ok &= abs(api.me_eval(a2, c2, z) - exact) < 1e-6
        zt = 0.875 + 0.625j
        b = api.m2l(a2, c2, zt)
        errs.append(abs(api.l2p(b, zt, z) - exact))
    ok &= errs[2] < 1e-10 and errs[0] > errs[1] > errs[2] or errs[2] < 1e-14
    return bool(ok)


def pin_fmm_converges(api):
    rng = np.random.default_rng(5)
    n = 1500
    x, y, q = rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1, 1, n)
    x[:500] = 0.6 + 0.02 * rng.standard_normal(500)
    y[:500] = 0.4 + 0.02 * rng.standard_normal(500)
    d = api.direct(x, y, q)
    e = [np.linalg.norm(api.fmm(x, y, q, (0.0, 0.0, 1.0), 4, p) - d) / np.linalg.norm(d)
         for p in (6, 12, 24, 32)]
    return e[0] > e[1] > e[2] and e[3] < 1e-12


PINS = [pin_ring_direct, pin_scaling, pin_gradient_vs_vortex, pin_ring_multipole,
        pin_ring_m2m_m2l, pin_fmm_converges]


@pytest.fixture(scope="module")
def api():
    import oracle
    return Api(_bind(ctypes.CDLL(oracle.build())))


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_laplace_pins(api, pin):
    assert pin(api)


def test_laplace_fmm_targets_match_full_run():
    import oracle
    rng = np.random.default_rng(6)
    n = 3000
    x, y, q = rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(-1, 1, n)
    full = oracle.laplace_fmm(x, y, q, (0, 0, 1), 5, 12)
    tg = np.array([0, 17, 1234, n - 1])
    part = oracle.laplace_fmm(x, y, q, (0, 0, 1), 5, 12, targets=tg)
    assert np.array_equal(part, full[tg])
    phi, me, le = oracle.laplace_fmm(x, y, q, (0, 0, 1), 3, 8, export=True)
    # the root's monopole term is the total charge
    assert abs(me[0, 0] - q.sum()) < 1e-12


# --- planted mistakes ---------------------------------------------------------------------

MUTANTS = {
    "p2m_no_1_over_k": ("            a[k] -= pw / (double)k;", "            a[k] -= pw;"),
    "m2m_log_term_sign": ("        cplx s = -a[0] * dpow[l] / (double)l;\n        for (int k = 1; k <= l; ++k) s += binom(l - 1",
                          "        cplx s = a[0] * dpow[l] / (double)l;\n        for (int k = 1; k <= l; ++k) s += binom(l - 1"),
    "m2m_binomial": ("s += binom(l - 1, k - 1) * a[k] * dpow[l - k];", "s += binom(l, k) * a[k] * dpow[l - k];"),
    "m2l_log_term_sign": ("        cplx s = -a[0] * ipow[m] / (double)m;", "        cplx s = a[0] * ipow[m] / (double)m;"),
    "m2l_binomial": ("binom(m + k - 1, k - 1) * a[k] * ipow[k + m];", "binom(m + k, k) * a[k] * ipow[k + m];"),
    "m2l_alternation": ("s += ((k % 2) ? -1.0 : 1.0) * binom(m + k - 1", "s += ((k % 2) ? 1.0 : -1.0) * binom(m + k - 1"),
    "m2l_constant_dropped": ("    cplx s0 = a[0] * clog(-d);", "    cplx s0 = 0.0;"),
    "direct_half_dropped": ("            s += q[j] * 0.5 * log(r2);", "            s += q[j] * log(r2);"),
    "near_half_dropped": ("                        nf += q[j] * 0.5 * log(r2);", "                        nf += q[j] * log(r2);"),
    "far_imaginary_part": ("double s = creal(l2p(p, le + (level_offset(L) + m) * p, zl, x[i] + I * y[i]));",
                           "double s = cimag(l2p(p, le + (level_offset(L) + m) * p, zl, x[i] + I * y[i]));"),
}


def _compile(text, tag):
    d = tempfile.mkdtemp(prefix=f"orclap_{tag}_")
    c, so = os.path.join(d, "o.c"), os.path.join(d, "o.so")
    open(c, "w").write(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", c, "-o",
                    so, "-lm"], check=True, capture_output=True)
    return Api(_bind(ctypes.CDLL(so)))


def test_unmutated_copy_passes_every_pin():
    api = _compile(open(SRC).read(), "clean")
    assert all(pin(api) for pin in PINS)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_mutant_fails_a_pin(name):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    api = _compile(src.replace(old, new), name)
    assert not all(pin(api) for pin in PINS), name
