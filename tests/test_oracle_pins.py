"""Pins for the FP64 oracle, against facts the paper and the mathematics fix
(closed forms, invariants, exact identities, brute force, convergence), so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails one of them.  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from conftest import rel_l2
from paper_0905_2637_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- kernel (Eq. 5, 7, 8)

def test_kernel_far_field_is_point_vortex(orc):
    # Eq. 7: a unit point vortex at the origin seen from (r, 0) moves the
    # fluid in +y at 1/(2 pi r); from (0, r) in -x.  Far from the core Eq. 8
    # must reduce to it.
    sigma, r = 1e-3, 0.1
    ku, kv = orc.kernel_sigma(r, 0.0, sigma)
    assert ku == 0.0 and kv == pytest.approx(1.0 / (2 * math.pi * r), rel=1e-15)
    ku, kv = orc.kernel_sigma(0.0, r, sigma)
    assert kv == 0.0 and ku == pytest.approx(-1.0 / (2 * math.pi * r), rel=1e-15)


@pytest.mark.parametrize("r_over_sigma", [0.01, 0.3, 1.0, 2.5, 7.0])
def test_kernel_matches_stokes_circulation_of_gaussian_blob(orc, r_over_sigma):
    # The Gaussian blob of Eq. 5 carries vorticity zeta_sigma; by Stokes the
    # azimuthal speed at radius r is (circulation inside r) / (2 pi r).  The
    # circulation is integrated numerically from Eq. 5 alone.
    sigma = 0.02
    r = r_over_sigma * sigma
    circ, _ = integrate.quad(
        lambda s: math.exp(-s * s / (2 * sigma * sigma)) / (2 * math.pi * sigma ** 2) * 2 * math.pi * s,
        0.0, r, epsabs=0, epsrel=1e-13)
    ut = circ / (2 * math.pi * r)
    ang = 0.7
    dx, dy = r * math.cos(ang), r * math.sin(ang)
    ku, kv = orc.kernel_sigma(dx, dy, sigma)
    # tangential component equals ut, radial component is zero
    assert (-math.sin(ang) * ku + math.cos(ang) * kv) == pytest.approx(ut, rel=1e-12)
    assert abs(math.cos(ang) * ku + math.sin(ang) * kv) < 1e-15 * abs(ut) + 1e-300


def test_kernel_core_is_solid_body_rotation(orc):
    # r << sigma: the blob's core rotates rigidly at angular speed 1/(4 pi sigma^2).
    sigma = 0.01
    for r in (1e-6, 1e-5):
        ku, kv = orc.kernel_sigma(r, 0.0, sigma)
        # next term of the series is -r^2 / (4 sigma^2) relative
        assert kv == pytest.approx(r / (4 * math.pi * sigma ** 2), rel=r * r / sigma ** 2)
        assert ku == 0.0


def test_kernel_self_is_zero(orc):
    assert orc.kernel_sigma(0.0, 0.0, 0.1) == (0.0, 0.0)


# ---------------------------------------------------------------- O1 direct sum (Eq. 9)

def test_direct_equilateral_triangle_rotates_rigidly(orc):
    # Three equal blobs at the corners of an equilateral triangle of side d:
    # by symmetry each moves perpendicular to its radius with speed
    # 2 cos(30 deg) * gamma * (1 - exp(-d^2 / 2 sigma^2)) / (2 pi d).
    d, sigma, gam = 0.3, 0.2, 0.7
    R = d / math.sqrt(3.0)
    ang = np.array([0.1, 0.1 + 2 * math.pi / 3, 0.1 + 4 * math.pi / 3])
    x, y = 0.4 + R * np.cos(ang), 0.5 + R * np.sin(ang)
    g = np.full(3, gam)
    u, v = orc.direct(x, y, g, sigma)
    speed = math.sqrt(3.0) * gam * (1 - math.exp(-d * d / (2 * sigma * sigma))) / (2 * math.pi * d)
    for i in range(3):
        rx, ry = x[i] - 0.4, y[i] - 0.5
        assert (-ry * u[i] + rx * v[i]) / R == pytest.approx(speed, rel=1e-13)
        assert abs(rx * u[i] + ry * v[i]) / R < 1e-15


def test_direct_invariants(orc):
    # K is odd and perpendicular to its argument, so sum gamma u = sum gamma v
    # = 0 and sum gamma (x u + y v) = 0 (linear impulse / no self-stretch).
    w = W.uniform(n=600, seed=3, sigma=0.02)
    u, v = orc.direct(w.x, w.y, w.gamma, w.sigma)
    scale = np.sum(np.abs(w.gamma) * np.hypot(u, v))
    assert abs(np.sum(w.gamma * u)) < 1e-13 * scale
    assert abs(np.sum(w.gamma * v)) < 1e-13 * scale
    assert abs(np.sum(w.gamma * (w.x * u + w.y * v))) < 1e-13 * scale


def test_direct_coincident_pair_contributes_nothing(orc):
    x = np.array([0.2, 0.2, 0.7])
    y = np.array([0.3, 0.3, 0.1])
    g = np.array([1.0, -2.0, 0.5])
    u, v = orc.direct(x, y, g, 0.05)
    u2, v2 = orc.direct(x[[0, 2]], y[[0, 2]], g[[0, 2]], 0.05)
    assert u[0] == u2[0] and v[0] == v2[0]


def test_direct_lamb_oseen(orc):
    # Sec. 7.1: lattice blobs (h / sigma = 0.8) carrying the Lamb-Oseen
    # vorticity of Eq. 16.  Eq. 17 as printed is garbled; the Lamb-Oseen
    # velocity is u_theta = Gamma0 / (2 pi r) (1 - exp(-r^2 / 4 nu t)).  The
    # blob sum is that field for the vorticity smoothed by the Gaussian basis,
    # whose variance adds: 4 nu t -> 4 nu t + 2 sigma^2.
    w = W.lamb_oseen()
    tg = W.sample_targets(w.n, 300, seed=11)
    u, v = orc.direct(w.x, w.y, w.gamma, w.sigma, targets=tg)
    x, y = w.x[tg], w.y[tg]
    r = np.hypot(x, y)
    m = r > 1e-9
    ut = (-y * u + x * v)[m] / r[m]
    ur = (x * u + y * v)[m] / r[m]
    eff = 0.1 ** 2 + 2 * w.sigma ** 2
    an = (1 - np.exp(-r[m] ** 2 / eff)) / (2 * math.pi * r[m])
    assert np.max(np.abs(ut - an)) < 1e-9 * np.max(an)
    assert np.max(np.abs(ur)) < 1e-9 * np.max(an)


# ---------------------------------------------------------------- tree (Sec. 2.1, 5.1)

def _interleave_by_strings(ix, iy, L):
    bx = format(ix, f"0{L}b") if L else ""
    by = format(iy, f"0{L}b") if L else ""
    s = "".join(b + a for a, b in zip(bx, by))  # most significant pair first: (iy_b, ix_b)
    return int(s, 2) if s else 0


def test_morton_matches_digit_interleave(orc):
    rng = np.random.default_rng(0)
    for L in (1, 3, 10, 15):
        for _ in range(50):
            ix, iy = (int(v) for v in rng.integers(0, 1 << L, 2))
            assert orc.morton(ix, iy, L) == _interleave_by_strings(ix, iy, L)


def test_binning_boundaries(orc):
    L, dom = 3, (0.0, 0.0, 1.0)
    x = np.array([0.0, 1.0, 0.125, np.nextafter(0.125, 0.0), 0.5, 0.999999])
    y = np.array([0.0, 1.0, 0.25, 0.25, np.nextafter(0.5, 1.0), 0.0])
    ix, iy, key = orc.bin(x, y, dom, L)
    assert list(ix) == [0, 7, 1, 0, 4, 7]
    assert list(iy) == [0, 7, 2, 2, 4, 0]
    assert all(k == orc.morton(a, b, L) for a, b, k in zip(ix, iy, key))
    for bad in (np.nextafter(1.0, 2.0), -1e-300, np.nan):
        with pytest.raises(orc.OracleError) as e:
            orc.bin(np.array([0.5, bad]), np.array([0.5, 0.5]), dom, L)
        assert e.value.code == orc.ORC_EDOMAIN


def test_binning_shifted_domain(orc):
    dom = (-2.0, 3.0, 4.0)  # [-2, 2] x [3, 7]
    ix, iy, _ = orc.bin(np.array([-2.0, 2.0, 0.0]), np.array([3.0, 7.0, 5.0]), dom, 2)
    assert list(ix) == [0, 3, 2] and list(iy) == [0, 3, 2]


def test_sort_is_stable_and_ranges_match(orc):
    w = W.tiny(5000, seed=2, L=4, clustered_frac=0.4)
    _, _, key = orc.bin(w.x, w.y, w.domain, w.L)
    perm, start = orc.sort(key, w.L)
    assert np.array_equal(perm, np.argsort(key, kind="stable").astype(np.uint32))
    assert np.array_equal(start, np.searchsorted(np.sort(key), np.arange((1 << 8) + 1)).astype(np.uint32))


def _golden_counts():
    per, cum = {}, {}
    with open(os.path.join(GOLDEN, "interaction_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "cum":
                cum[int(parts[1])] = (int(parts[2]), int(parts[3]))
            else:
                per[int(parts[0])] = int(parts[2])
    return per, cum


def test_interaction_list_counts_match_golden(orc):
    per, cum = _golden_counts()
    for l in range(2, 7):
        n = 1 << l
        total = sum(len(orc.interaction_list(l, ix, iy)) for ix in range(n) for iy in range(n))
        assert total == per[l]
    for L, (pairs, lam) in cum.items():
        assert sum(per[l] for l in range(2, L + 1)) == pairs
        assert ((4 ** (L + 1)) - 1) // 3 == lam


def test_interaction_list_membership(orc):
    # Every member is well separated from the box (Chebyshev distance >= 2)
    # and its parent is adjacent to the box's parent; every such box is a
    # member; interior boxes have exactly 27 (Table 1); output is in ascending
    # Morton order of the source.
    for l in (2, 3, 4):
        n = 1 << l
        for ix in range(n):
            for iy in range(n):
                il = orc.interaction_list(l, ix, iy)
                got = {(int(a), int(b)) for a, b in il}
                want = {(sx, sy) for sx in range(n) for sy in range(n)
                        if max(abs(sx - ix), abs(sy - iy)) >= 2
                        and max(abs(sx // 2 - ix // 2), abs(sy // 2 - iy // 2)) <= 1}
                assert got == want
                keys = [orc.morton(a, b, l) for a, b in il]
                assert keys == sorted(keys)
                if 2 <= ix // 2 * 2 and ix // 2 + 1 < n // 2 and 2 <= iy // 2 * 2 and iy // 2 + 1 < n // 2:
                    assert len(il) == 27
    assert orc.interaction_list(1, 0, 1).shape == (0, 2)


# ---------------------------------------------------------------- expansions

def _cluster(seed, n, c, rad):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * math.pi, n)
    rr = rad * np.sqrt(rng.uniform(0, 1, n))
    return c.real + rr * np.cos(ang), c.imag + rr * np.sin(ang), rng.uniform(-1, 1, n)


def _cauchy(x, y, g, z):
    return np.sum(g / (z - (x + 1j * y)))


def test_p2m_series_converges_to_cauchy_sum(orc):
    zc = 0.3 + 0.2j
    x, y, g = _cluster(1, 40, zc, 0.1)
    z = 0.9 - 0.1j  # |z - zc| / radius ratio ~ 6.7
    exact = _cauchy(x, y, g, z)
    rho = 0.1 / abs(z - zc)
    prev = None
    for p in (2, 4, 8, 16):
        a = orc.p2m(x, y, g, zc, p)
        err = abs(orc.me_eval(a, zc, z) - exact)
        bound = np.sum(np.abs(g)) * rho ** p / (abs(z - zc) - 0.1)
        assert err <= bound * 1.0000001
        if prev is not None:
            assert err < prev
        prev = err
    a0 = orc.p2m(x, y, g, zc, 1)
    assert a0[0] == pytest.approx(np.sum(g), rel=1e-14)


def test_m2m_is_exact_recentering(orc):
    zp = 0.5 + 0.5j
    p = 14
    total = np.zeros(p, complex)
    xs, ys, gs = [], [], []
    for c, off in enumerate([-0.125 - 0.125j, 0.125 - 0.125j, -0.125 + 0.125j, 0.125 + 0.125j]):
        zc = zp + off
        x, y, g = _cluster(10 + c, 25, zc, 0.1)
        xs.append(x); ys.append(y); gs.append(g)
        total += orc.m2m(orc.p2m(x, y, g, zc, p), zc, zp)
    direct = orc.p2m(np.concatenate(xs), np.concatenate(ys), np.concatenate(gs), zp, p)
    assert np.max(np.abs(total - direct)) < 1e-13 * np.max(np.abs(direct))


def test_m2l_converges_geometrically(orc):
    zs, zt = 0.0 + 0.0j, 3.0 + 1.0j  # box centres two to three widths apart
    x, y, g = _cluster(5, 30, zs, 0.5)
    z = zt + 0.3 - 0.2j
    exact = _cauchy(x, y, g, z)
    errs = []
    for p in (4, 8, 12, 16, 20):
        b = orc.m2l(orc.p2m(x, y, g, zs, p), zs, zt)
        errs.append(abs(orc.l2p(b, zt, z) - exact) / abs(exact))
    assert errs[-1] < 1e-8
    for a, b in zip(errs, errs[1:]):
        assert b < a


def test_l2l_is_exact_recentering(orc):
    rng = np.random.default_rng(4)
    p = 15
    b = rng.standard_normal(p) + 1j * rng.standard_normal(p)
    zp, zc = 0.5 + 0.5j, 0.25 + 0.75j
    bc = orc.l2l(b, zp, zc)
    for z in (0.3 + 0.7j, 0.2 + 0.8j, 0.26 + 0.74j):
        w1 = orc.l2p(b, zp, z)
        w2 = orc.l2p(bc, zc, z)
        assert abs(w1 - w2) < 1e-14 * np.sum(np.abs(b))


def test_l2p_of_m2l_matches_singular_velocity_sign(orc):
    # A single vortex far away: the LE evaluated at the target reproduces
    # u = Im(w) / 2pi, v = Re(w) / 2pi of the Eq. 7 point vortex.
    g0, zs, zt = 1.3, 0.0j, 4.0 + 0.0j
    b = orc.m2l(np.array([g0] + [0.0] * 11, complex), zs, zt)
    w = orc.l2p(b, zt, zt)
    u, v = w.imag / (2 * math.pi), w.real / (2 * math.pi)
    assert u == pytest.approx(0.0, abs=1e-16) and v == pytest.approx(g0 / (2 * math.pi * 4.0), rel=1e-14)


# ---------------------------------------------------------------- O2 and O3

def test_substituted_equals_direct_for_tiny_blobs(orc):
    # With sigma far below the leaf width, every far pair has
    # exp(-r^2 / 2 sigma^2) < 1e-80, so kernel substitution changes nothing.
    w = W.tiny(800, seed=5, L=3, sigma=0.004)
    u1, v1 = orc.direct(w.x, w.y, w.gamma, w.sigma)
    u2, v2 = orc.substituted(w.x, w.y, w.gamma, w.domain, w.L, w.sigma)
    assert rel_l2(u2, v2, u1, v1) < 1e-14


def test_substituted_differs_for_wide_blobs_and_keeps_invariants(orc):
    w = W.tiny(800, seed=6, L=4, sigma=0.05)
    u1, v1 = orc.direct(w.x, w.y, w.gamma, w.sigma)
    u2, v2 = orc.substituted(w.x, w.y, w.gamma, w.domain, w.L, w.sigma)
    assert rel_l2(u2, v2, u1, v1) > 1e-3  # Type I error is visible here
    scale = np.sum(np.abs(w.gamma) * np.hypot(u2, v2))
    assert abs(np.sum(w.gamma * u2)) < 1e-13 * scale
    assert abs(np.sum(w.gamma * (w.x * u2 + w.y * v2))) < 1e-13 * scale


def test_fmm_level_one_equals_direct(orc):
    # L = 1: all four leaves are mutual neighbours, nothing is far.
    w = W.tiny(700, seed=8, L=1, p=6, sigma=0.03)
    u1, v1 = orc.direct(w.x, w.y, w.gamma, w.sigma)
    u3, v3 = orc.fmm(w.x, w.y, w.gamma, w.domain, 1, 6, w.sigma)
    assert rel_l2(u3, v3, u1, v1) < 1e-14


@pytest.mark.parametrize("L", [2, 3, 4])
def test_fmm_converges_to_substituted_sum(orc, L):
    w = W.tiny(1500, seed=9 + L, L=L, clustered_frac=0.3)
    u2, v2 = orc.substituted(w.x, w.y, w.gamma, w.domain, L, w.sigma)
    errs = []
    for p in (4, 8, 12, 16, 24, 32):
        u3, v3 = orc.fmm(w.x, w.y, w.gamma, w.domain, L, p, w.sigma)
        errs.append(rel_l2(u3, v3, u2, v2))
    # worst-case contraction per term for this separation is sqrt(2)/(4-sqrt(2))
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.547 ** 3
    assert errs[-1] < 1e-11


def test_fmm_target_subset_matches_full(orc):
    w = W.tiny(3000, seed=21, L=4, p=10, clustered_frac=0.2)
    u, v = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    tg = W.sample_targets(w.n, 97, seed=3)
    us, vs = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, targets=tg)
    assert np.array_equal(us, u[tg]) and np.array_equal(vs, v[tg])


def test_fmm_exported_expansions_are_consistent(orc):
    w = W.tiny(2000, seed=22, L=3, p=9)
    u, v, me, le = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, export=True)
    ix, iy, key = orc.bin(w.x, w.y, w.domain, w.L)
    off = ((1 << (2 * w.L)) - 1) // 3
    r = 1.0 / (1 << w.L)
    for m in (0, 5, 37, 63):
        sel = key == m
        bx, by = int(ix[sel][0]) if sel.any() else 0, int(iy[sel][0]) if sel.any() else 0
        if not sel.any():
            assert np.all(me[off + m] == 0)
            continue
        zc = (bx + 0.5) * r + 1j * (by + 0.5) * r
        a = orc.p2m(w.x[sel], w.y[sel], w.gamma[sel], zc, w.p)
        assert np.max(np.abs(me[off + m] - a)) < 1e-14 * np.max(np.abs(a))
    # root ME's zeroth coefficient is the total circulation
    assert me[0, 0] == pytest.approx(np.sum(w.gamma), rel=1e-12)
    # levels 0 and 1 receive no local expansion
    assert np.all(le[:5] == 0)


def test_fmm_is_thread_count_independent(orc):
    w = W.tiny(2500, seed=23, L=3, p=8)
    u1, v1 = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, nthreads=1)
    u4, v4 = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, nthreads=4)
    assert np.array_equal(u1, u4) and np.array_equal(v1, v4)


def test_fmm_rejects_bad_arguments(orc):
    w = W.tiny(10, seed=1)
    with pytest.raises(orc.OracleError):
        orc.fmm(w.x, w.y, w.gamma, w.domain, 3, 0, w.sigma)
    with pytest.raises(orc.OracleError):
        orc.fmm(w.x, w.y, w.gamma, w.domain, 3, 5, -1.0)
    with pytest.raises(orc.OracleError) as e:
        orc.fmm(w.x + 2.0, w.y, w.gamma, w.domain, 3, 5, w.sigma)
    assert e.value.code == orc.ORC_EDOMAIN
