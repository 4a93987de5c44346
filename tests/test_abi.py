"""The C-ABI library: it loads, exports every symbol include/petfmm.h
declares, and its host-side logic (argument checks, interaction-list table,
work-model level choice, memory estimate) behaves.  No GPU needed."""
import ctypes
import math

import numpy as np
import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = lib.header_symbols()
    assert len(names) >= 20
    handle = lib.load()
    for n in names:
        assert hasattr(handle, n), n


def test_strerror_names_every_code(lib):
    seen = set()
    for code in range(0, -8, -1):
        s = lib.petfmm_strerror(code)
        assert s and s != "unknown status"
        seen.add(s)
    assert len(seen) == 8
    assert lib.petfmm_strerror(-99) == "unknown status"


@pytest.mark.parametrize("args", [
    ((0.0, 0.0, 0.0), 4, 8, 0.01),     # zero width
    ((0.0, 0.0, 1.0), 0, 8, 0.01),     # L < 1
    ((0.0, 0.0, 1.0), 16, 8, 0.01),    # L > 15
    ((0.0, 0.0, 1.0), 4, 0, 0.01),     # p < 1
    ((0.0, 0.0, 1.0), 4, 41, 0.01),    # p > 40
    ((0.0, 0.0, 1.0), 4, 8, 0.0),      # sigma <= 0
    ((0.0, float("nan"), 1.0), 4, 8, 0.01),
])
def test_create_rejects_bad_arguments_before_touching_cuda(lib, args):
    with pytest.raises(lib.PetfmmError) as e:
        lib.petfmm_create(*args, lib.PETFMM_MIXED, lib.PETFMM_F32, None)
    assert e.value.code == lib.PETFMM_EINVAL


def test_create_rejects_bad_modes(lib):
    for prec, dt in ((2, 0), (0, 2), (-1, 0)):
        with pytest.raises(lib.PetfmmError) as e:
            lib.petfmm_create((0, 0, 1), 4, 8, 0.01, prec, dt, None)
        assert e.value.code == lib.PETFMM_EINVAL


def test_interaction_list_matches_oracle(lib, orc):
    # Same sets as the oracle's own construction (Sec. 2.2, Table 1); the
    # library lists them in its kernel order, the oracle in Morton order.
    for level in (2, 3, 5):
        n = 1 << level
        rng = np.random.default_rng(level)
        boxes = [(0, 0), (n - 1, n - 1), (0, n - 1), (1, 2)] + [tuple(rng.integers(0, n, 2)) for _ in range(30)]
        for ix, iy in boxes:
            a = lib.petfmm_debug_interaction_list(level, int(ix), int(iy))
            b = orc.interaction_list(level, int(ix), int(iy))
            assert sorted(map(tuple, a)) == sorted(map(tuple, b))
    assert lib.petfmm_debug_interaction_list(1, 0, 0).shape == (0, 2)
    with pytest.raises(lib.PetfmmError):
        lib.petfmm_debug_interaction_list(3, 8, 0)


def test_choose_levels_respects_kernel_substitution_guard(lib):
    dom = (0.0, 0.0, 1.0)
    for n in (1_000, 46_000, 262_144, 4_000_000):
        sigma = 0.5 / math.sqrt(n)
        L = lib.petfmm_choose_levels(n, 12, sigma, dom)
        assert 1 <= L <= 12
        r = 1.0 / (1 << L)
        assert math.exp(-r * r / (2 * sigma * sigma)) <= 1e-8
    # more particles never want a shallower tree (same sigma)
    Ls = [lib.petfmm_choose_levels(n, 12, 1e-4, dom) for n in (1e3, 1e4, 1e5, 1e6, 1e7)]
    assert Ls == sorted(Ls)
    with pytest.raises(lib.PetfmmError):
        lib.petfmm_choose_levels(100, 0, 0.01, dom)


def test_serve_estimate_grows_with_problem(lib):
    a = lib.petfmm_serve_estimate_bytes(1_000_000, 8, 17, lib.PETFMM_MIXED)
    b = lib.petfmm_serve_estimate_bytes(4_000_000, 10, 17, lib.PETFMM_MIXED)
    c = lib.petfmm_serve_estimate_bytes(4_000_000, 10, 17, lib.PETFMM_FP64)
    assert 0 < a < b < c
    # a 4M-blob, L = 10, p = 17 request fits a 150 GB budget more than 100 times
    assert 150e9 / b > 100
    assert lib.petfmm_serve_estimate_bytes(-1, 8, 17, 1) == 0


def test_missing_library_fails_loudly(monkeypatch, lib):
    import importlib
    mod = importlib.import_module("paper_0905_2637_gb300._lib")
    monkeypatch.setattr(mod, "_lib", None)
    monkeypatch.setattr(mod, "LIB_PATH", "/nonexistent/libpetfmm.so")
    with pytest.raises(ImportError):
        mod.load()


def test_checked_build_exists_and_reports_itself(lib):
    """The bounds-checked variant is built beside the library; its
    petfmm_debug_checks answers 3 (files checked), the regular one 0."""
    import ctypes
    import os
    from paper_0905_2637_gb300 import build as b
    assert os.path.exists(b.LIB_CHECKED)
    lines = (ctypes.c_uint32 * 3)()
    assert lib.load().petfmm_debug_checks(lines) == 0 and list(lines) == [0, 0, 0]
    chk = ctypes.CDLL(b.LIB_CHECKED)
    chk.petfmm_debug_checks.restype = ctypes.c_int
    chk.petfmm_debug_checks.argtypes = [ctypes.c_void_p]
    assert chk.petfmm_debug_checks(lines) == 3
    assert chk.petfmm_debug_checks(None) == lib.PETFMM_EINVAL


@pytest.mark.parametrize("args", [
    ((0.0, 0.0, 0.0, 1.0), 0, 8),       # L < 1
    ((0.0, 0.0, 0.0, 1.0), 9, 8),       # L > 8
    ((0.0, 0.0, 0.0, 1.0), 3, 0),       # p < 1
    ((0.0, 0.0, 0.0, 1.0), 3, 17),      # p > 16
    ((0.0, 0.0, 0.0, 0.0), 3, 8),       # W <= 0
    ((0.0, float("inf"), 0.0, 1.0), 3, 8),
])
def test_create3d_rejects_bad_arguments_before_touching_cuda(lib, args):
    from paper_0905_2637_gb300 import fmm3d
    with pytest.raises(lib.PetfmmError) as e:
        fmm3d.petfmm3d_create(*args, lib.PETFMM_MIXED, lib.PETFMM_F32)
    assert e.value.code == lib.PETFMM_EINVAL
    for prec, dt in ((2, 0), (0, 2)):
        with pytest.raises(lib.PetfmmError):
            fmm3d.petfmm3d_create((0, 0, 0, 1), 3, 8, prec, dt)
