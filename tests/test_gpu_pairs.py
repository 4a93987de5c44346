"""The pairwise near field of the mixed path.

Every pair of blobs in the same leaf or in neighbouring leaves that both
hold at least 32 blobs is summed once: the kernel of Eq. 8 is odd in the
offset, so the velocity a blob b induces on a and the one a induces on b
share K(x_a - x_b) (Sec. 2.1, Eq. 9), and the reaction on the source travels
with it.  Heavy pairs are
cut into pieces along the target leaf (whole 128-target chunks, at most 256
tiles of 128 x 32 per piece), the source leaf's partial sums of pieces 1 ..
kept apart and added in piece order; when those partial sums would need more
than one scratch entry per blob, no pair is cut.

Against the directed evaluation of every ordered pair (PETFMM_OPT_P2P_PAIRS =
0) the result differs by FP32 rounding only: both sum the same FP32 terms in
other orders, and each stays within the mixed path's 1e-5 of the FP64 FMM, so
the two differ by at most 2e-5 (a dropped or doubled leaf pair shows at 1e-3
or more); the pairwise result's error is also no more than twice the directed
one's (plus 1e-6, for cases where both are tiny); and it is bitwise
reproducible (single-owner slots, fixed summation order)."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOLMX = 1e-5
TOLPAIR = 2e-5
FWD = ((1, 0), (-1, 1), (0, 1), (1, 1))


def leaf_grid(orc, w):
    """Blobs per leaf, [iy, ix], from the oracle's tree."""
    _, _, key = orc.bin(w.x, w.y, w.domain, w.L)
    _, start = orc.sort(key, w.L)
    cnt = np.diff(start.astype(np.int64))
    n = 1 << w.L
    grid = np.zeros((n, n), np.int64)
    for m in np.nonzero(cnt)[0]:
        ix = iy = 0
        for b in range(w.L):
            ix |= ((int(m) >> (2 * b)) & 1) << b
            iy |= ((int(m) >> (2 * b + 1)) & 1) << b
        grid[iy, ix] = cnt[m]
    return grid


def expected_pieces(grid):
    """(pair items, scratch entries wanted, unordered blob pairs) of the
    pairwise rule and the piece rule."""
    n = grid.shape[0]
    items = extra = sym = 0
    for iy in range(n):
        for ix in range(n):
            na = int(grid[iy, ix])
            if na < 32:
                continue
            items += 1                      # the leaf's own pairs
            sym += na * (na - 1) // 2
            for dx, dy in FWD:
                bx, by = ix + dx, iy + dy
                if not (0 <= bx < n and 0 <= by < n):
                    continue
                nb = int(grid[by, bx])
                if nb < 32:
                    continue
                ca, cb = -(-na // 128), -(-nb // 32)
                npc = min(ca, max(1, -(-(ca * cb) // 256)))
                per = -(-ca // npc)
                npc = -(-ca // per)
                items += npc
                extra += (npc - 1) * nb
                sym += na * nb
    return items, extra, sym


def run_ctx(w, precision, **opts):
    _lib = G.lib()
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision=precision, dtype=w.dtype)
    ctx.set_option(_lib.PETFMM_OPT_POISON, 1)
    ctx.set_option(_lib.PETFMM_OPT_TIMING, 1)
    for k, v in opts.items():
        ctx.set_option(getattr(_lib, "PETFMM_OPT_" + k), v)
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    u, v = ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    out = (u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64))
    st = ctx.stats()
    ctx.close()
    return out, st


@pytest.mark.parametrize("w", [
    W.tiny(60_000, 51, L=5, p=12, dtype="f32"),                        # ~59 per leaf, TPL 2
    W.tiny(200_000, 52, L=5, p=14, clustered_frac=0.3, dtype="f32"),   # 4 targets per lane
    W.tiny(40_000, 53, L=5, p=12, sigma=0.002, clustered_frac=0.3),    # exp branch, f64 I/O
    W.lattice(side=256, L=5, p=12, dtype="f32"),                       # 64 per leaf exactly
], ids=["uniform", "clustered", "general", "lattice"])
def test_pairwise_matches_directed_and_fp64(w):
    (u1, v1), st = run_ctx(w, "mixed", P2P_PAIRS=1)
    (u0, v0), _ = run_ctx(w, "mixed", P2P_PAIRS=0)
    (u64, v64), _ = run_ctx(w, "fp64")
    assert st["p2p_pair_items"] > 0
    assert np.all(np.isfinite(u1)) and np.all(np.isfinite(v1))
    assert G.rel_l2(u1, v1, u0, v0) <= TOLPAIR
    e1, e0 = G.rel_l2(u1, v1, u64, v64), G.rel_l2(u0, v0, u64, v64)
    assert e1 <= TOLMX and e0 <= TOLMX
    assert e1 <= 2.0 * e0 + 1e-6


def test_leaf_counts_around_the_thresholds(orc):
    # leaves of 0, 1, 31, 32, 33, 95, 96, 97, 128, 129 and 300 blobs in a
    # seeded arrangement: every mix of pairwise / directed neighbours and of
    # 2 / 4 targets per lane, ragged chunks on both sides
    rng = np.random.default_rng(61)
    L, n = 4, 16
    counts = rng.choice([0, 1, 31, 32, 33, 95, 96, 97, 128, 129, 300], size=(n, n))
    xs, ys = [], []
    for iy in range(n):
        for ix in range(n):
            c = int(counts[iy, ix])
            xs.append((ix + rng.uniform(0.02, 0.98, c)) / n)
            ys.append((iy + rng.uniform(0.02, 0.98, c)) / n)
    x, y = np.concatenate(xs), np.concatenate(ys)
    g = rng.uniform(-1.0, 1.0, x.size)
    w = W.Workload("thresholds", x.astype(np.float32), y.astype(np.float32),
                   g.astype(np.float32), 0.25 / n, W.UNIT_DOMAIN, L, 12, "f32")
    assert np.array_equal(leaf_grid(orc, w), counts)
    (u1, v1), st = run_ctx(w, "mixed", P2P_PAIRS=1)
    (u0, v0), _ = run_ctx(w, "mixed", P2P_PAIRS=0)
    items, extra, sym = expected_pieces(counts)
    assert st["p2p_pair_items"] == items and st["p2p_split_entries"] == extra
    assert st["p2p_sym_pairs"] == sym and 0.0 < st["pairs_load_balance"] <= 1.0
    assert G.rel_l2(u1, v1, u0, v0) <= TOLPAIR
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    assert G.rel_l2(u1, v1, ur, vr) <= TOLMX


def test_heavy_pairs_are_split_and_reproducible(orc):
    # a tight clump of 30 000 blobs among 570 000 uniform ones: 41 pairs of
    # clump leaves are cut into pieces, their scratch fits
    w = W.tiny(600_000, 41, L=7, p=12, clustered_frac=0.05, dtype="f32")
    items, extra, sym = expected_pieces(leaf_grid(orc, w))
    assert 0 < extra <= w.n
    (u1, v1), st = run_ctx(w, "mixed", P2P_PAIRS=1)
    assert st["p2p_pair_items"] == items and st["p2p_split_entries"] == extra
    assert st["p2p_sym_pairs"] == sym
    (u1b, v1b), _ = run_ctx(w, "mixed", P2P_PAIRS=1, P2P_MODE=1)
    assert np.array_equal(u1, u1b) and np.array_equal(v1, v1b)
    (u0, v0), _ = run_ctx(w, "mixed", P2P_PAIRS=0)
    assert G.rel_l2(u1, v1, u0, v0) <= TOLPAIR
    (u64, v64), _ = run_ctx(w, "fp64")
    e1, e0 = G.rel_l2(u1, v1, u64, v64), G.rel_l2(u0, v0, u64, v64)
    assert e1 <= TOLMX and e1 <= 2.0 * e0 + 1e-6
    tg = W.sample_targets(w.n, 300)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, targets=tg)
    assert G.rel_l2(u1[tg], v1[tg], ur, vr) <= TOLMX


def test_split_scratch_overflow_keeps_pairs_whole(orc):
    # two adjacent leaves of 20 000 blobs each: cutting their pairs would want
    # far more than one scratch entry per blob, so no pair is cut
    rng = np.random.default_rng(71)
    m = 20_000
    x = np.concatenate([rng.uniform(0.26, 0.49, m), rng.uniform(0.51, 0.74, m)])
    y = rng.uniform(0.51, 0.74, 2 * m)
    g = rng.uniform(-1.0, 1.0, 2 * m) / m
    w = W.Workload("two-leaves", x.astype(np.float32), y.astype(np.float32),
                   g.astype(np.float32), 0.01, W.UNIT_DOMAIN, 2, 12, "f32")
    items, extra, _ = expected_pieces(leaf_grid(orc, w))
    assert extra > w.n
    (u1, v1), st = run_ctx(w, "mixed", P2P_PAIRS=1)
    assert st["p2p_pair_items"] == items and st["p2p_split_entries"] == extra
    (u0, v0), _ = run_ctx(w, "mixed", P2P_PAIRS=0)
    assert G.rel_l2(u1, v1, u0, v0) <= TOLPAIR
    tg = W.sample_targets(w.n, 200)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, targets=tg)
    assert G.rel_l2(u1[tg], v1[tg], ur, vr) <= TOLMX
