"""The tree cut of Sec. 4 and the model of Sec. 5.1-5.2 (host code, no GPU):
subtree work against Eq. 13/14 written out, the communication model against
a count by enumeration of the interaction lists, and the z-order partition
against a brute-force search of every contiguous split."""
import itertools

import numpy as np
import pytest

import __graft_entry__


@pytest.fixture(scope="module")
def sh():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import shard
    return shard


def _morton(ix, iy):
    k = 0
    for b in range(16):
        k |= ((ix >> b) & 1) << (2 * b) | ((iy >> b) & 1) << (2 * b + 1)
    return k


def test_weights_are_eq13_for_inner_boxes_and_eq14_per_leaf(sh):
    L, k, p = 5, 2, 12
    rng = np.random.default_rng(1)
    counts = rng.integers(0, 40, 1 << (2 * L)).astype(np.uint32)
    w = sh.weights(L, k, p, counts)
    per = 1 << (2 * (L - k))
    inner = (per - 1) // 3
    for s in range(1 << (2 * k)):
        n = counts[s * per:(s + 1) * per].astype(np.float64)
        ref = inner * p * p * (2 * 4 + 27) + np.sum(2 * n * p + p * p * 27 + 9 * n * n)
        assert w[s] == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("L,k", [(7, 3), (6, 2), (4, 1)])
def test_comm_model_counts_the_interaction_list_boxes(sh, L, k):
    """Eq. 11 (both directions, lateral) and the corner count (diagonal) are
    the number of boxes one subtree's interaction lists take from the other."""
    side = 1 << k
    a = (side // 2 - 1, side // 2 - 1)
    lat, diag = sh.comm(L, k, alpha=1.0)
    for (dx, dy), model in (((1, 0), lat), ((1, 1), diag)):
        b = (a[0] + dx, a[1] + dy)
        if not (b[0] < side and b[1] < side):
            pytest.skip("cut too coarse for this neighbour")
        total = 0
        for src, dst in ((a, b), (b, a)):
            owner = np.ones(1 << (2 * k), np.int32)
            owner[_morton(*src)] = 0
            _, boxes = sh.halo(L, k, owner, 0)
            for lvl, m in boxes:
                sub = m >> (2 * (lvl - k))
                if sub == _morton(*dst):
                    total += 1
        assert total == model


def test_partition_is_contiguous_nonempty_and_optimal(sh):
    L, k, p = 4, 2, 8
    rng = np.random.default_rng(3)
    for trial in range(6):
        counts = (rng.pareto(1.2, 1 << (2 * L)) * 4).astype(np.uint32)
        w = sh.weights(L, k, p, counts)
        nsub = w.size
        for P in (1, 2, 3, 5):
            owner, summ = sh.partition(L, k, p, counts, P)
            assert np.all(np.diff(owner) >= 0) and owner[0] == 0 and owner[-1] == P - 1
            assert all(s["subtrees"] >= 1 for s in summ)
            best = min(max(w[a:b].sum() for a, b in zip((0,) + cuts, cuts + (nsub,)))
                       for cuts in itertools.combinations(range(1, nsub), P - 1))
            assert max(s["work"] for s in summ) == pytest.approx(best, rel=1e-9)
            for r, s in enumerate(summ):
                assert s["work"] == pytest.approx(w[owner == r].sum(), rel=1e-12)
                assert s["first_subtree"] == np.flatnonzero(owner == r)[0]
                assert s["last_subtree"] == np.flatnonzero(owner == r)[-1] + 1
                per = 1 << (2 * (L - k))
                assert s["particles"] == sum(int(counts[t * per:(t + 1) * per].sum())
                                             for t in np.flatnonzero(owner == r))


def test_partition_comm_is_the_model_over_cut_edges(sh):
    L, k, p, P = 6, 2, 10, 3
    counts = np.random.default_rng(5).integers(0, 30, 1 << (2 * L)).astype(np.uint32)
    owner, summ = sh.partition(L, k, p, counts, P)
    lat, diag = sh.comm(L, k)
    side = 1 << k
    ref = np.zeros(P)
    for sy in range(side):
        for sx in range(side):
            s = _morton(sx, sy)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    nx, ny = sx + dx, sy + dy
                    if (dx or dy) and 0 <= nx < side and 0 <= ny < side:
                        t = _morton(nx, ny)
                        if owner[t] != owner[s]:
                            ref[owner[s]] += diag if (dx and dy) else lat
    assert np.allclose([s["comm"] for s in summ], ref)


def test_halo_leaves_are_the_foreign_neighbours(sh):
    L, k = 4, 1
    owner = np.array([0, 1, 1, 0], np.int32)
    leaves, _ = sh.halo(L, k, owner, 0)
    lo = sh.leaf_owner(L, k, owner)
    side = 1 << L
    ref = set()
    for y in range(side):
        for x in range(side):
            if lo[_morton(x, y)] != 0:
                continue
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if 0 <= x + dx < side and 0 <= y + dy < side:
                        m = _morton(x + dx, y + dy)
                        if lo[m] != 0:
                            ref.add(m)
    assert set(leaves.tolist()) == ref


def test_bad_arguments(sh):
    from paper_0905_2637_gb300 import _lib
    with pytest.raises(_lib.PetfmmError):
        sh.partition(4, 2, 8, np.zeros(1 << 8, np.uint32), 17)   # more ranks than subtrees
    with pytest.raises(_lib.PetfmmError):
        sh.comm(3, 4)                                             # cut below the leaves
