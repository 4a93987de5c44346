"""The host-built translation operators (no GPU).  The FP64 M2M, L2L and M2L
tables (Sec. 2.2, rescaled coefficients) that both precisions use equal the
oracle's translations applied to unit coefficients, for both kernels and
p = 1 .. 40.  The tensor-core M2L's images: hi + lo of every image
reproduces the oracle's M2L operator for each of the 40 offsets; hi holds
TF32 values (low 13 mantissa bits zero), lo the remainder, and the padding
is zero.  The block images put each target class's operator in its own
column block, bit for bit the per-offset image, and zeros where the class's
offset is within one box."""
import numpy as np
import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


# the 40 offsets delta of [-3, 3]^2 minus [-1, 1]^2, row by row
OFFSETS = [(dx, dy) for dy in range(-3, 4) for dx in range(-3, 4) if max(abs(dx), abs(dy)) >= 2]


def dims(p):
    k2 = 2 * p
    return k2, (k2 + 7) & ~7, (k2 + 15) & ~15, (k2 + 7) & ~7   # K2, Kpad, Npad, NW


def unpack(img, kpad, ncol):
    """[k / 4][n][k % 4] -> B[k][n]"""
    return img.reshape(kpad // 4, ncol, 4).transpose(0, 2, 1).reshape(kpad, ncol)


def oracle_b(orc, p, delta, kernel):
    """B = [[Re T, Im T], [-Im T, Re T]], T[k][m]: LE coefficient m produced by
    the unit ME coefficient k of a source box at offset delta (width 1)."""
    m2l = orc.lap_m2l if kernel else orc.m2l
    t = np.zeros((p, p), complex)
    for k in range(p):
        e = np.zeros(p, complex)
        e[k] = 1.0
        t[k] = m2l(e, complex(*delta), 0.0)
    return np.block([[t.real, t.imag], [-t.imag, t.real]])


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("p", [1, 5, 8, 12, 17, 24])
def test_row_images_match_the_oracle_operators(lib, orc, p, kernel):
    k2, kpad, npad, _ = dims(p)
    img = lib.petfmm_debug_m2l_images(p, kernel, 0)
    slot = kpad * npad
    assert img.size == 40 * 2 * slot
    for o, delta in enumerate(OFFSETS):
        hi_raw = img[(2 * o) * slot:(2 * o + 1) * slot]
        assert np.all(hi_raw.view(np.uint32) & 0x1FFF == 0)
        hi = unpack(hi_raw, kpad, npad).astype(np.float64)
        lo = unpack(img[(2 * o + 1) * slot:(2 * o + 2) * slot], kpad, npad).astype(np.float64)
        b = hi + lo
        ref = oracle_b(orc, p, delta, kernel)
        # hi + lo carries the FP64 value to about 2^-35 (lo is FP32 too)
        assert np.allclose(b[:k2, :k2], ref, rtol=1e-9, atol=1e-30), (delta, kernel)
        assert not np.any(b[k2:, :]) and not np.any(b[:, k2:])
        # lo is what hi leaves of the FP32 value
        assert np.all(np.abs(lo) <= np.abs(hi) * 2.0 ** -10 + 1e-38)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("p", [3, 8, 17, 24])
def test_block_images_put_the_four_classes_side_by_side(lib, p, kernel):
    k2, kpad, npad, nw = dims(p)
    rows = lib.petfmm_debug_m2l_images(p, kernel, 0)
    blocks = lib.petfmm_debug_m2l_images(p, kernel, 1)
    slot, bslot = kpad * npad, kpad * 4 * nw
    assert blocks.size == 36 * 2 * bslot
    index = {d: o for o, d in enumerate(OFFSETS)}
    for cs in range(4):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                g = cs * 9 + (dy + 1) * 3 + dx + 1
                for hl in range(2):
                    bimg = unpack(blocks[(2 * g + hl) * bslot:(2 * g + hl + 1) * bslot], kpad, 4 * nw)
                    for c in range(4):
                        d = (2 * dx + (cs & 1) - (c & 1), 2 * dy + (cs >> 1) - (c >> 1))
                        col = bimg[:, c * nw:(c + 1) * nw]
                        if max(abs(d[0]), abs(d[1])) < 2:
                            assert not np.any(col)
                            continue
                        o = index[d]
                        rimg = unpack(rows[(2 * o + hl) * slot:(2 * o + hl + 1) * slot], kpad, npad)
                        assert np.array_equal(col.view(np.uint32), rimg[:, :nw].view(np.uint32))


def test_every_class_gets_its_27_operators(lib):
    # over the 36 (source class, dy, dx) images, each target class meets each
    # of its 27 interaction-list offsets exactly once
    for c in range(4):
        seen = []
        for cs in range(4):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    d = (2 * dx + (cs & 1) - (c & 1), 2 * dy + (cs >> 1) - (c >> 1))
                    if max(abs(d[0]), abs(d[1])) >= 2:
                        seen.append(d)
        assert len(seen) == 27 == len(set(seen))
        ix, iy = 10 + (c & 1), 10 + (c >> 1)
        il = lib.petfmm_debug_interaction_list(6, ix, iy)
        assert sorted(seen) == sorted((int(a) - ix, int(b) - iy) for a, b in il)


def test_bad_arguments(lib):
    for args in ((0, 0, 0), (25, 0, 0), (8, 2, 0), (8, 0, 2)):
        with pytest.raises(lib.PetfmmError):
            lib.petfmm_debug_m2l_images(*args)


# ---- the FP64 operator tables behind both precisions ----------------------

@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("p", [1, 4, 12, 17, 30, 40])
def test_m2m_l2l_m2l_tables_match_the_oracle(lib, orc, p, kernel):
    """Rescaled coefficients at child width 1 (parent width 2): M2M maps a
    child's a~_k to its parent's a~'_l = a'_l / 2^l; L2L maps the parent's
    scaled LE (unscaled b_m = 2^-(m+1) c^_m, Laplace 2^-m) to the child's;
    M2L maps a~_k at offset delta to c^_m at box width 1."""
    m2m = orc.lap_m2m if kernel else orc.m2m
    m2l = orc.lap_m2l if kernel else orc.m2l
    M = lib.petfmm_debug_op_table(p, kernel, 0)
    L = lib.petfmm_debug_op_table(p, kernel, 1)
    T = lib.petfmm_debug_op_table(p, kernel, 2)
    assert M.shape == L.shape == (4, p, p) and T.shape == (40, p, p)
    scale_le = 2.0 ** -(np.arange(p) + (0 if kernel else 1))
    for c in range(4):
        e = complex((c & 1) - 0.5, (c >> 1) - 0.5)
        for k in range(p):
            unit = np.zeros(p, complex)
            unit[k] = 1.0
            ref = m2m(unit, e, 0.0) / 2.0 ** np.arange(p)
            assert np.allclose(M[c, :, k], ref, rtol=1e-12, atol=1e-300), ("M2M", c, k)
            ref = orc.l2l(unit * scale_le, 0.0, e)
            assert np.allclose(L[c, :, k], ref, rtol=1e-12, atol=1e-300), ("L2L", c, k)
    for o, delta in enumerate(OFFSETS):
        for k in range(p):
            unit = np.zeros(p, complex)
            unit[k] = 1.0
            ref = m2l(unit, complex(*delta), 0.0)
            assert np.allclose(T[o, k], ref, rtol=1e-12, atol=1e-300), ("M2L", delta, k)


def test_op_table_bad_arguments(lib):
    for args in ((0, 0, 0), (41, 0, 0), (8, 2, 0), (8, 0, 3)):
        with pytest.raises(lib.PetfmmError):
            lib.petfmm_debug_op_table(*args)
