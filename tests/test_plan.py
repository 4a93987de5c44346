"""Host-side launch planning of batches (no GPU): every launch's tasks are a
contiguous block-ordered slice, and every instance, level and tree sweep is
covered exactly once -- the kernels binary-search their block in that slice."""
import math

import numpy as np
import pytest

import __graft_entry__
from paper_0905_2637_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


UNITS_PER_BLOCK = {0: 1024, 1: 256, 2: 256, 3: 256, 4: 256, 5: 32, 6: 1, 7: 1, 70: 1, 71: 1, 72: 1,
                   73: 1}


def _instances(seed, k):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(0, 50_000)) if i % 5 else 0
        out.append(dict(domain=(0.0, 0.0, 1.0), levels=int(rng.integers(1, 11)), order=int(rng.choice([8, 12, 17, 30])),
                        sigma=1e-3, n=n))
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seed,k", [(1, 1), (2, 7), (3, 64), (4, 200)])
def test_plan_ranges_are_contiguous_and_complete(lib, precision, seed, k):
    insts = _instances(seed, k)
    # tensor-core blocks at levels 5 to 7 only when the plan has >= 512 of them
    # at those levels
    blocks = sum((2 ** (l - 1) // 8) * (2 ** (l - 1) // 16)
                 for it in insts if it["order"] <= 24 for l in range(5, min(it["levels"], 7) + 1))
    use_blocks = precision == 1 and blocks >= 512
    plan = lib.petfmm_debug_plan(precision, insts)
    ranges = {}
    for row in plan:
        ranges.setdefault(int(row[0]), []).append(row)
    # each range appears as one contiguous run in launch order
    ids = [int(r[0]) for r in plan]
    runs = [ids[0]] + [b for a, b in zip(ids, ids[1:]) if a != b]
    assert len(runs) == len(set(runs))
    for rid, rows in ranges.items():
        rows = np.array(rows)
        per = UNITS_PER_BLOCK.get(rid, 256)
        blocks = np.ceil(rows[:, 3] / per).astype(np.int64)
        assert rows[0, 4] == 0
        assert np.array_equal(rows[1:, 4], np.cumsum(blocks)[:-1])
        assert np.all(rows[:, 3] > 0)
    for i, it in enumerate(insts):
        L, p, n = it["levels"], it["order"], it["n"]
        for rid in (0, 2):
            rows = [r for r in ranges.get(rid, []) if r[1] == i]
            assert (len(rows) == 1 and rows[0][3] == n) if n else not rows
        for rid, units in ((1, 4 ** L + 1), (3, 4 ** L), (4, 4 ** L)):
            rows = [r for r in ranges[rid] if r[1] == i]
            assert len(rows) == 1 and rows[0][3] == units
        simt = sorted(int(r[2]) for r in ranges.get(5, []) if r[1] == i)
        tc = sorted(int(r[2]) for r in ranges.get(6, []) if r[1] == i)
        # every level has a SIMT launch; the levels with >= 128 parent cells per
        # row (mixed path, p <= 24) also get the tensor-core launch in blocks,
        # one CTA per 8 x 16 parent cells (all four classes), which takes the
        # dense units; levels 5 to 7 too when the plan has >= 512 blocks.  (The
        # row units, launch 6, run only with PETFMM_OPT_TC_BLOCKS = 2.)
        assert simt == list(range(2, L + 1))
        assert tc == []
        tcb = sorted(int(r[2]) for r in ranges.get(7, []) if r[1] == i)
        assert tcb == ([l for l in range(5 if use_blocks else 8, L + 1)]
                       if precision == 1 and p <= 24 else [])
        for r in ranges.get(7, []):
            if r[1] == i:
                w = 2 ** (int(r[2]) - 1)
                assert r[3] == (w // 8) * (w // 16)
        # the other levels of the mixed path (p <= 24) get the tiled SIMT
        # launch, one CTA per (class, 128 target boxes: a 128-cell segment of
        # a parent row, or several whole rows where rows are shorter)
        # (one launch per order class, p <= 8, 12, 18, 24: ids 70 .. 73)
        cls = 70 + (0 if p <= 8 else 1 if p <= 12 else 2 if p <= 18 else 3)
        tile_rows = [r for rid in range(70, 74) for r in ranges.get(rid, []) if r[1] == i]
        assert all(r[0] == cls for r in tile_rows)
        tile = sorted(int(r[2]) for r in tile_rows)
        assert tile == ([l for l in range(2, L + 1) if l not in tc and l not in tcb]
                        if precision == 1 and p <= 24 else [])
        for r in tile_rows:
            if r[1] == i:
                w = 2 ** (int(r[2]) - 1)
                seg = min(w, 128)
                rows = max(1, min(64 // seg, w)) if w < 128 else 1
                assert r[3] == 4 * (w // rows) * (w // seg)
        m2m = [(rid, int(r[2])) for rid, rs in ranges.items() if 100 <= rid < 200 for r in rs if r[1] == i]
        assert sorted(l for _, l in m2m) == list(range(2, L))
        # bottom-up: round r holds level L - 1 - r
        assert all(l == L - 1 - (rid - 100) for rid, l in m2m)
        l2l = [(rid, int(r[2])) for rid, rs in ranges.items() if rid >= 200 for r in rs if r[1] == i]
        assert sorted(l for _, l in l2l) == list(range(3, L + 1))
        assert all(l == 3 + (rid - 200) for rid, l in l2l)
        for rid, l in m2m + l2l:
            row = [r for r in ranges[rid] if r[1] == i][0]
            assert row[3] == 4 ** l * p


def test_plan_rejects_too_many_key_bits(lib):
    insts = [dict(domain=(0, 0, 1), levels=15, order=8, sigma=1e-3, n=10)] * 8
    with pytest.raises(lib.PetfmmError):
        lib.petfmm_debug_plan(1, insts)


def test_automatic_levels_in_plan_match_choose_levels(lib):
    ws = W.batch(n_inst=12, seed=2)
    insts = [dict(domain=w.domain, levels=0, order=w.p, sigma=w.sigma, n=w.n) for w in ws]
    plan = lib.petfmm_debug_plan(1, insts)
    for i, w in enumerate(ws):
        L = lib.petfmm_choose_levels(w.n, w.p, w.sigma, w.domain)
        row = [r for r in plan if r[0] == 3 and r[1] == i][0]
        assert row[3] == 4 ** L
        assert math.exp(-(1.0 / 2 ** L) ** 2 / (2 * w.sigma ** 2)) <= 1e-8
