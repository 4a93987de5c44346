"""Pins of the 3D oracle (the octree extension of Sec. 8; oracle3d.c), each
against something other than the oracle's own formulas: closed forms of the
1/r kernel, a library's Legendre functions, exactness of the recentring
operators, the partition of every pair into near field and interaction
lists, brute force on tiny inputs, and geometric convergence of the FMM to
the direct sum."""
import itertools
import math

import numpy as np
import pytest

import oracle as O

P_SH = 12


def _rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def test_regular_harmonics_match_library_legendre():
    """R_n^m(v) = r^n P_n^m(cos t) e^{i m phi} / (n + m)! with P_n^m without
    the Condon-Shortley phase, against scipy's associated Legendre function
    (which carries the phase)."""
    sp = pytest.importorskip("scipy.special")
    v = np.array([0.31, -0.52, 0.27])
    r = np.linalg.norm(v)
    ct, ph = v[2] / r, math.atan2(v[1], v[0])
    R, Iv = O.harmonics3d(v, P_SH)
    for n in range(P_SH):
        for m in range(0, n + 1):
            leg = sp.lpmv(m, n, ct) * (-1) ** m
            want_r = r ** n * leg * np.exp(1j * m * ph) / math.factorial(n + m)
            want_i = math.factorial(n - m) * leg * np.exp(1j * m * ph) / r ** (n + 1)
            assert R[n, P_SH - 1 + m] == pytest.approx(want_r, rel=1e-12, abs=1e-300)
            assert Iv[n, P_SH - 1 + m] == pytest.approx(want_i, rel=1e-12)
            if m:
                assert R[n, P_SH - 1 - m] == pytest.approx((-1) ** m * np.conj(want_r), rel=1e-12)
                assert Iv[n, P_SH - 1 - m] == pytest.approx((-1) ** m * np.conj(want_i), rel=1e-12)


def test_addition_theorem_gives_inverse_distance():
    """1/|x - y| = sum conj(R(y)) I(x) for |y| < |x|: the series converges
    geometrically in |y|/|x| to the closed form."""
    x = np.array([1.1, -0.4, 0.8])
    y = np.array([0.2, 0.25, -0.15])
    want = 1.0 / np.linalg.norm(x - y)
    errs = []
    for P in (6, 12, 24):
        Ry, _ = O.harmonics3d(y, P)
        _, Ix = O.harmonics3d(x, P)
        s = sum(np.conj(Ry[n, P - 1 + m]) * Ix[n, P - 1 + m]
                for n in range(P) for m in range(-n, n + 1))
        assert abs(s.imag) < 1e-14
        errs.append(abs(s.real - want) / want)
    ratio = np.linalg.norm(y) / np.linalg.norm(x)
    assert errs[2] < 1e-13 and errs[0] < 2 * ratio ** 6 and errs[1] < 2 * ratio ** 12


def test_derivative_identities_by_finite_differences():
    P, h = 9, 1e-5
    v = np.array([0.3, -0.2, 0.45])
    R0, _ = O.harmonics3d(v, P, irregular=False)

    def d(ax):
        e = np.zeros(3)
        e[ax] = h
        return (O.harmonics3d(v + e, P, False)[0] - O.harmonics3d(v - e, P, False)[0]) / (2 * h)
    gx, gy, gz = d(0), d(1), d(2)

    def get(n, m):
        return R0[n, P - 1 + m] if 0 <= n and abs(m) <= n else 0.0
    for n in range(1, P):
        for m in range(-n, n + 1):
            assert abs(gz[n, P - 1 + m] - get(n - 1, m)) < 1e-9
            assert abs(gx[n, P - 1 + m] - 1j * gy[n, P - 1 + m] - get(n - 1, m - 1)) < 1e-9
            assert abs(gx[n, P - 1 + m] + 1j * gy[n, P - 1 + m] + get(n - 1, m + 1)) < 1e-9


def test_direct_sum_brute_force_and_closed_forms():
    # two unit charges one apart: phi = 1, |E| = 1 along the axis
    phi, ex, ey, ez = O.direct3d([0.0, 1.0], [0.0, 0.0], [0.0, 0.0], [1.0, 2.0])
    assert phi[0] == pytest.approx(2.0) and phi[1] == pytest.approx(1.0)
    assert ex[0] == pytest.approx(-2.0) and ex[1] == pytest.approx(1.0)
    assert ey[0] == 0.0 and ez[1] == 0.0
    # five charges by hand-written loops; a coincident pair contributes 0
    rng = np.random.default_rng(3)
    x, y, z = rng.random((3, 5))
    x[4], y[4], z[4] = x[1], y[1], z[1]
    q = rng.uniform(-1, 1, 5)
    phi, ex, ey, ez = O.direct3d(x, y, z, q)
    for i in range(5):
        p_ = e_ = 0.0
        e_ = np.zeros(3)
        for j in range(5):
            dvec = np.array([x[i] - x[j], y[i] - y[j], z[i] - z[j]])
            r = np.linalg.norm(dvec)
            if r == 0:
                continue
            p_ += q[j] / r
            e_ += q[j] * dvec / r ** 3
        assert phi[i] == pytest.approx(p_, rel=1e-14)
        assert np.allclose([ex[i], ey[i], ez[i]], e_, rtol=1e-13, atol=1e-13)


def test_direct_field_obeys_newtons_third_law():
    rng = np.random.default_rng(4)
    x, y, z = rng.random((3, 400))
    q = rng.uniform(-1, 1, 400)
    _, ex, ey, ez = O.direct3d(x, y, z, q)
    scale = np.sum(np.abs(q[:, None] * np.stack([ex, ey, ez], 1)))
    for e in (ex, ey, ez):
        assert abs(np.sum(q * e)) < 1e-13 * scale


def test_multipole_expansion_converges_to_the_direct_potential():
    rng = np.random.default_rng(5)
    c = np.array([0.5, 0.5, 0.5])
    pts = c + (rng.random((40, 3)) - 0.5) * 0.25
    q = rng.uniform(-1, 1, 40)
    far = np.array([2.1, -0.7, 1.3])
    want = np.sum(q / np.linalg.norm(far - pts, axis=1))
    errs = [abs(O.me_eval3d(O.p2m3d(*pts.T, q, c, p), c, far, p) - want) / abs(want)
            for p in (2, 6, 10, 14)]
    assert errs[-1] < 1e-12 and all(b < a for a, b in zip(errs, errs[1:]))


def test_m2m_is_exact():
    """P2M about a child centre shifted by M2M equals P2M about the parent."""
    rng = np.random.default_rng(6)
    cc = np.array([0.25, 0.75, 0.25])
    cp = np.array([0.5, 0.5, 0.5])
    pts = cc + (rng.random((30, 3)) - 0.5) * 0.5
    q = rng.uniform(-1, 1, 30)
    for p in (1, 5, 11):
        a = O.m2m3d(O.p2m3d(*pts.T, q, cc, p), cc, cp, p)
        b = O.p2m3d(*pts.T, q, cp, p)
        assert np.max(np.abs(a - b)) < 1e-14 * np.max(np.abs(b))


def test_l2l_is_exact_and_l2p_field_is_minus_the_gradient():
    """A local expansion is a polynomial: recentred by L2L it gives the same
    potential and field everywhere; the field of L2P is -grad of its
    potential (central differences)."""
    rng = np.random.default_rng(7)
    p = 9
    Lc = np.zeros(p * (2 * p - 1), np.complex128)
    for n in range(p):
        Lc[O.idx3(p, n, 0)] = rng.normal()
        for m in range(1, n + 1):
            a = complex(rng.normal(), rng.normal())
            Lc[O.idx3(p, n, m)] = a
            Lc[O.idx3(p, n, -m)] = (-1) ** m * np.conj(a)   # a real potential
    c = np.array([0.5, 0.5, 0.5])
    cc = np.array([0.6, 0.4, 0.55])
    L2 = O.l2l3d(Lc, c, cc, p)
    h = 1e-5
    for pt in rng.random((5, 3)):
        a = O.l2p3d(Lc, c, pt, p)
        b = O.l2p3d(L2, cc, pt, p)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            fd = (O.l2p3d(Lc, c, pt + e, p)[0] - O.l2p3d(Lc, c, pt - e, p)[0]) / (2 * h)
            assert a[1 + ax] == pytest.approx(-fd, rel=1e-6, abs=1e-8)


def test_m2l_converges_to_the_direct_potential_and_field():
    rng = np.random.default_rng(8)
    cs = np.array([0.125, 0.125, 0.125])
    ct = np.array([0.625, 0.375, 0.125])     # two boxes of width 1/4 apart
    src = cs + (rng.random((50, 3)) - 0.5) * 0.25
    q = rng.uniform(-1, 1, 50)
    tgt = ct + (rng.random(3) - 0.5) * 0.25
    d = tgt - src
    r = np.linalg.norm(d, axis=1)
    want = np.array([np.sum(q / r), *np.sum(q[:, None] * d / r[:, None] ** 3, 0)])
    errs = []
    for p in (4, 8, 12, 16):
        got = np.array(O.l2p3d(O.m2l3d(O.p2m3d(*src.T, q, cs, p), cs, ct, p), ct, tgt, p))
        errs.append(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    assert errs[-1] < 1e-5 and all(b < a for a, b in zip(errs, errs[1:]))


def test_interaction_lists_and_near_field_cover_every_pair_once():
    """For leaves t, s of a level-3 octree, exactly one of: s is a neighbour
    of t, or some level l >= 2 has ancestor(s) in IL(ancestor(t)) -- the
    partition of the sum that makes the FMM equal the direct sum."""
    L = 3
    side = 1 << L
    il = {}
    for l in range(2, L + 1):
        n = 1 << l
        for ix, iy, iz in itertools.product(range(n), repeat=3):
            il[(l, ix, iy, iz)] = {tuple(r) for r in O.interaction_list3d(l, ix, iy, iz)}
    sizes = [len(v) for (l, *_), v in il.items() if l == 3]
    # interior 6^3 - 3^3; a box at (1, 1, 1) of level 3 (parent in a corner): 4^3 - 3^3
    assert max(sizes) == 189 and min(sizes) == 37
    for t in itertools.product(range(side), repeat=3):
        for s in itertools.product(range(side), repeat=3):
            near = all(abs(a - b) <= 1 for a, b in zip(t, s))
            far = sum(tuple(c >> (L - l) for c in s) in il[(l, *(c >> (L - l) for c in t))]
                      for l in range(2, L + 1))
            assert near + far == 1


def test_morton_bin_and_sort_by_brute_force():
    rng = np.random.default_rng(9)
    L = 3
    x, y, z = rng.random((3, 500))
    x[0], y[1], z[2] = 1.0, 0.0, 1.0       # closed cube: boundary points
    key = O.bin3d(x, y, z, (0.0, 0.0, 0.0, 1.0), L)
    for i in range(500):
        b = [min(int(np.floor(v * 8)), 7) for v in (x[i], y[i], z[i])]
        k = 0
        for bit in range(L):
            for d in range(3):
                k |= ((b[d] >> bit) & 1) << (3 * bit + d)
        assert key[i] == k == O.morton3d(*b, L)
    perm, start = O.sort3d(key, L)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(start, np.searchsorted(np.sort(key), np.arange(8 ** L + 1)))
    with pytest.raises(O.OracleError):
        O.bin3d([1.5], [0.5], [0.5], (0.0, 0.0, 0.0, 1.0), L)


def test_fmm_without_far_field_is_the_direct_sum():
    """L = 1: every leaf is a neighbour of every other, the interaction lists
    are empty, and the FMM is the direct sum to rounding."""
    rng = np.random.default_rng(10)
    x, y, z = rng.random((3, 700))
    q = rng.uniform(-1, 1, 700)
    a = O.fmm3d(x, y, z, q, (0, 0, 0, 1), 1, 6)
    b = O.direct3d(x, y, z, q)
    for u, v in zip(a, b):
        assert _rel(u, v) < 1e-14


def test_fmm_converges_geometrically_to_the_direct_sum():
    rng = np.random.default_rng(11)
    n = 4000
    x, y, z = rng.random((3, n))
    x[:1000] = 0.3 + 0.05 * rng.standard_normal(1000).clip(-5, 5)   # a cluster
    q = rng.uniform(-1, 1, n)
    ref = O.direct3d(x, y, z, q)
    errs = []
    for p in (3, 6, 9, 12):
        got = O.fmm3d(x, y, z, q, (0, 0, 0, 1), 3, p)
        errs.append(max(_rel(got[0], ref[0]), _rel(np.stack(got[1:]), np.stack(ref[1:]))))
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-5
    # Newton's third law holds for the FMM to its truncation error
    got = O.fmm3d(x, y, z, q, (0, 0, 0, 1), 3, 12)
    for e in got[1:]:
        assert abs(np.sum(q * e)) < 1e-5 * np.sum(np.abs(q * e))


def test_bench_interaction_pair_count_is_the_enumeration():
    """The 3D bench leg's algorithmic M2L pair count (a closed form that
    factors per axis) against the oracle's interaction lists."""
    import bench
    for L in (2, 3):
        tot = 0
        for l in range(2, L + 1):
            n = 1 << l
            for ix, iy, iz in itertools.product(range(n), repeat=3):
                tot += len(O.interaction_list3d(l, ix, iy, iz))
        assert bench._il_pairs3(L) == tot
