"""Instrumentation: per-stage timings (the per-stage breakdown of Fig. 6),
pair counts against the oracle's tree, the load-balance metric of Eq. 20,
launch counting, and the host-array entry point."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_stage_times_and_counters(orc):
    _lib = G.lib()
    w = W.tiny(50_000, 3, L=6, p=12, clustered_frac=0.4)
    keep = []
    G.run(w, "mixed", timing=True, ctx_out=keep)
    ctx = keep[0]
    t = ctx.stage_times()
    assert set(t) == set(_lib.STAGES) and all(v >= 0 for v in t.values())
    st = ctx.stats()
    # ordered near-field pairs, counted from the oracle's own tree
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
    pad = np.pad(grid, 1)
    near = sum(pad[1 + dy:1 + dy + n, 1 + dx:1 + dx + n] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    assert st["p2p_pairs"] == int(np.sum(grid * (near - 1) * (grid > 0)))
    assert st["m2l_pairs"] == sum((6 * (1 << l) - 8) ** 2 - (3 * (1 << l) - 2) ** 2 for l in range(2, w.L + 1))
    assert 0.0 < st["p2p_load_balance"] <= 1.0
    assert st["kernel_launches"] > 10 and st["evaluations"] == 1
    ctx.close()


def test_evaluate_host_matches_device_path():
    _lib = G.lib()
    w = W.tiny(20_000, 4, L=5, p=12, dtype="f32")
    ud, vd = G.run(w, "mixed")
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype="f32")
    uh, vh = ctx.evaluate_host(w.x, w.y, w.gamma)
    ctx.close()
    assert np.array_equal(uh.astype(np.float64), ud) and np.array_equal(vh.astype(np.float64), vd)


def test_repeated_evaluations_are_deterministic():
    _lib = G.lib()
    w = W.tiny(100_000, 5, L=7, p=17, clustered_frac=0.5, dtype="f32")
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype="f32")
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    outs = []
    for _ in range(3):
        u, v = ctx.evaluate(x, y, g)
        ctx.sync()
        outs.append((u.cpu().numpy(), v.cpu().numpy()))
    ctx.close()
    for u, v in outs[1:]:
        assert np.array_equal(u, outs[0][0]) and np.array_equal(v, outs[0][1])


def test_reused_context_matches_fresh_context():
    # A context keeps its buffers between evaluations; a second, different
    # problem must not see anything of the first (no stale expansions).
    _lib = G.lib()
    a = W.tiny(40_000, 21, L=6, p=12, clustered_frac=0.6)
    b = W.tiny(30_000, 22, L=6, p=12, clustered_frac=0.2)
    ctx = _lib.Context(a.domain, 6, 12, a.sigma, precision="mixed", dtype="f64")
    for w in (a, b):
        x, y, g = G.to_dev((w.x, w.y, w.gamma))
        u, v = ctx.evaluate(x, y, g)
        assert ctx.sync() == 0
    u, v = u.cpu().numpy(), v.cpu().numpy()
    ctx.close()
    uf, vf = G.run(b, "mixed", poison=False)
    assert np.array_equal(u, uf) and np.array_equal(v, vf)


def test_p2p_dispatch_order_does_not_change_results():
    # each target's sum runs in one lane in a fixed source order, so taking
    # the work items heaviest first (mode 0) or in leaf order (mode 1) gives
    # the same bits, in both precisions
    _lib = G.lib()
    cases = [(W.tiny(60_000, 21, L=6, p=12, clustered_frac=0.7, dtype="f32"), "mixed"),
             # sigma small against the leaf: the exp-branch kernel, whose
             # tiers are chosen by warp votes
             (W.tiny(40_000, 24, L=5, p=12, sigma=0.002, clustered_frac=0.3), "mixed"),
             (W.tiny(30_000, 22, L=5, p=14, clustered_frac=0.7), "fp64"),
             (W.tiny(1, 23, L=3, p=8), "mixed")]
    for w, prec in cases:
        outs = []
        for mode in (0, 1):
            ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision=prec, dtype=w.dtype)
            ctx.set_option(_lib.PETFMM_OPT_P2P_MODE, mode)
            ctx.set_option(_lib.PETFMM_OPT_POISON, 1)
            x, y, g = G.to_dev((w.x, w.y, w.gamma))
            u, v = ctx.evaluate(x, y, g)
            assert ctx.sync() == 0
            outs.append((u.cpu().numpy(), v.cpu().numpy()))
            ctx.close()
        assert np.all(np.isfinite(outs[0][0])) and np.all(np.isfinite(outs[0][1]))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_graph_replay_matches_plain_launches():
    # PETFMM_OPT_GRAPH: the launch sequence is captured once per launch shape
    # and replayed; new caller arrays of the same shape reuse the graph (the
    # plan is read from device memory), a new size captures again.  Results
    # are bitwise those of plain launches.
    _lib = G.lib()
    torch = G.torch_cuda()
    w1 = W.tiny(50_000, 31, L=6, p=12, clustered_frac=0.5, dtype="f32")
    w2 = W.tiny(50_000, 32, L=6, p=12, clustered_frac=0.5, dtype="f32")
    w3 = W.tiny(20_000, 33, L=6, p=12, clustered_frac=0.5, dtype="f32")
    ref = {}
    plain = _lib.Context(w1.domain, w1.L, w1.p, w1.sigma, precision="mixed", dtype="f32")
    for w in (w1, w2, w3):
        x, y, g = G.to_dev((w.x, w.y, w.gamma))
        u, v = plain.evaluate(x, y, g)
        assert plain.sync() == 0
        ref[w.name + str(w.n) + str(w.x[0])] = (u.cpu().numpy(), v.cpu().numpy())
    plain.close()
    ctx = _lib.Context(w1.domain, w1.L, w1.p, w1.sigma, precision="mixed", dtype="f32")
    ctx.set_option(_lib.PETFMM_OPT_GRAPH, 1)
    ctx.set_option(_lib.PETFMM_OPT_TIMING, 1)
    for w in (w1, w1, w2, w3, w1):
        x, y, g = G.to_dev((w.x, w.y, w.gamma))
        u, v = ctx.evaluate(x, y, g)
        assert ctx.sync() == 0
        ur, vr = ref[w.name + str(w.n) + str(w.x[0])]
        assert np.array_equal(u.cpu().numpy(), ur) and np.array_equal(v.cpu().numpy(), vr)
        st = ctx.stage_times()
        assert st["p2p"] > 0 and all(t >= 0 for t in st.values())
    assert ctx.stats()["kernel_launches"] > 0
    ctx.close()
    torch.cuda.synchronize()


def test_overlap_streams_match_one_stream():
    # PETFMM_OPT_OVERLAP: the expansion chain on the context's second stream,
    # beside the near field, plain and captured in a graph, gives bitwise the
    # velocities of one stream; the stage times stay readable.
    _lib = G.lib()
    torch = G.torch_cuda()
    w = W.tiny(60_000, 41, L=6, p=12, clustered_frac=0.5, dtype="f32")
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    outs = []
    for overlap, graph in ((0, 0), (1, 0), (1, 1), (0, 1)):
        ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype="f32")
        ctx.set_option(_lib.PETFMM_OPT_OVERLAP, overlap)
        ctx.set_option(_lib.PETFMM_OPT_GRAPH, graph)
        ctx.set_option(_lib.PETFMM_OPT_TIMING, 1)
        for _ in range(2):
            u, v = ctx.evaluate(x, y, g)
            assert ctx.sync() == 0
        st = ctx.stage_times()
        assert st["m2l"] > 0 and st["pairs"] > 0 and all(t >= 0 for t in st.values())
        outs.append((u.cpu().numpy(), v.cpu().numpy()))
        ctx.close()
    for u, v in outs[1:]:
        assert np.array_equal(u, outs[0][0]) and np.array_equal(v, outs[0][1])
    torch.cuda.synchronize()
