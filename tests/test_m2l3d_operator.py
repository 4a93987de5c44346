"""The 3D mixed path's M2L operators (the real p^2 x p^2 matrices the library
builds on the host, fmm3d.cu) against the 3D oracle's M2L: for every input
basis vector of the real coefficient basis, the oracle's translation of the
corresponding real-potential multipole expansion, read back in the same
basis, is the matrix column.  Host code only."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def f3():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0905_2637_gb300 import fmm3d
    return fmm3d


def _basis(p):
    """(coefficient (n, m), part) of each real index."""
    re = [(n, m) for n in range(p) for m in range(n + 1)]
    im = [(n, m) for n in range(p) for m in range(1, n + 1)]
    return [(nm, 0) for nm in re] + [(nm, 1) for nm in im]


@pytest.mark.parametrize("p,delta", [(4, (2, 0, 0)), (6, (-3, 2, 1)), (8, (2, -2, 3)),
                                     (8, (0, 0, -2)), (11, (3, 3, 3))])
def test_operator_columns_are_the_oracle_translation(f3, p, delta):
    a = f3.m2l_operator(p, *delta)
    basis = _basis(p)
    assert a.shape == (p * p, p * p) == (len(basis), len(basis))
    cs, ct = np.zeros(3), np.array(delta, dtype=np.float64)
    for k, ((n, m), part) in enumerate(basis):
        M = np.zeros(p * (2 * p - 1), np.complex128)
        v = 1.0 if part == 0 else 1j
        M[O.idx3(p, n, m)] = v
        if m:
            M[O.idx3(p, n, -m)] = (-1) ** m * np.conj(v)   # a real potential
        Lc = O.m2l3d(M, cs, ct, p)
        col = np.array([Lc[O.idx3(p, nn, mm)].real if pt == 0 else Lc[O.idx3(p, nn, mm)].imag
                        for (nn, mm), pt in basis])
        scale = max(1.0, np.max(np.abs(col)))
        assert np.max(np.abs(a[k] - col)) <= 1e-12 * scale, (k, n, m, part)
        # the Im of m = 0 outputs, which the basis leaves out, is zero
        for nn in range(p):
            assert abs(Lc[O.idx3(p, nn, 0)].imag) <= 1e-12 * scale


def test_bad_offsets_are_rejected(f3):
    from paper_0905_2637_gb300 import _lib
    for d in ((1, 1, 0), (4, 0, 0), (0, 0, 0)):
        with pytest.raises(_lib.PetfmmError):
            f3.m2l_operator(8, *d)
    with pytest.raises(_lib.PetfmmError):
        f3.m2l_operator(17, 2, 0, 0)


def _real_series(p, n, m, part):
    """The real-potential series of one basis vector (oracle storage)."""
    S = np.zeros(p * (2 * p - 1), np.complex128)
    v = 1.0 if part == 0 else 1j
    S[O.idx3(p, n, m)] = v
    if m:
        S[O.idx3(p, n, -m)] = (-1) ** m * np.conj(v)
    return S


def _read_real(p, S, basis):
    return np.array([S[O.idx3(p, n, m)].real if pt == 0 else S[O.idx3(p, n, m)].imag
                     for (n, m), pt in basis])


@pytest.mark.parametrize("p", [1, 3, 8, 10])
@pytest.mark.parametrize("kind", ["m2m", "l2l"])
def test_shift_operator_columns_are_the_oracle_translation(f3, p, kind):
    # child width 1, parent width 2 centred at the origin; the scaled series
    # are M~ = M / w^n and L~ = L w^(n+1) with each box's own width w
    basis = _basis(p)
    deg = np.array([n for (n, _), _ in basis], dtype=np.float64)
    code = f3.PETFMM3D_SHIFT_M2M if kind == "m2m" else f3.PETFMM3D_SHIFT_L2L
    for octant in range(8):
        a = f3.shift_operator(p, code, octant)
        assert a.shape == (p * p, p * p)
        cc = np.array([0.5 if octant & (1 << ax) else -0.5 for ax in range(3)])
        for k, ((n, m), part) in enumerate(basis):
            S = _real_series(p, n, m, part)
            if kind == "m2m":
                out = O.m2m3d(S, cc, np.zeros(3), p)
                col = _read_real(p, out, basis) / 2.0 ** deg
            else:
                Sp = S / 2.0 ** (n + 1)       # the parent's unscaled local expansion
                out = O.l2l3d(Sp, np.zeros(3), cc, p)
                col = _read_real(p, out, basis)
            scale = max(1.0, np.max(np.abs(col)))
            assert np.max(np.abs(a[k] - col)) <= 1e-12 * scale, (octant, k, n, m, part)


def test_shift_operator_bad_arguments(f3):
    from paper_0905_2637_gb300 import _lib
    for args in ((8, 2, 0), (8, -1, 0), (8, 0, 8), (8, 1, -1), (0, 0, 0), (17, 0, 0)):
        with pytest.raises(_lib.PetfmmError):
            f3.shift_operator(*args)
