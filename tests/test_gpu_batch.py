"""Batched evaluation: many instances of uneven size in one pass; each
instance's result is bit-for-bit what it gets alone, and matches the oracle."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(ctx, ws, levels):
    torch = G.torch_cuda()
    insts, outs = [], []
    for w, L in zip(ws, levels):
        x, y, g = G.to_dev((w.x, w.y, w.gamma))
        u = torch.empty_like(x)
        v = torch.empty_like(x)
        insts.append(dict(domain=w.domain, levels=L, order=w.p, sigma=w.sigma, x=x, y=y, gamma=g, u=u, v=v))
        outs.append((u, v))
    ctx.evaluate_batch(insts)
    assert ctx.sync() == 0
    return [(u.cpu().numpy(), v.cpu().numpy()) for u, v in outs]


@pytest.mark.parametrize("precision,blocks", [("fp64", 0), ("mixed", 0), ("mixed", 1)])
def test_batch_equals_alone_bitwise(orc, precision, blocks):
    # (blocks = 1: tensor-core blocks at levels 5 to 7 in the batch and alone)
    _lib = G.lib()
    ws = W.batch(n_inst=24, seed=4, n_min=200, n_max=40_000)
    levels = [_lib.petfmm_choose_levels(w.n, w.p, w.sigma, w.domain) for w in ws]
    ctx = _lib.Context((0, 0, 1), 2, 8, 0.01, precision=precision, dtype="f64")
    ctx.set_option(_lib.PETFMM_OPT_TC_BLOCKS, blocks)
    res = _batch(ctx, ws, [0] * len(ws))  # automatic L inside the library
    ctx.close()
    for w, L, (u, v) in zip(ws, levels, res):
        ua, va = G.run(w, precision, L=L, options={_lib.PETFMM_OPT_TC_BLOCKS: blocks})
        assert np.array_equal(u, ua) and np.array_equal(v, va)
    # spot-check a few instances against the oracle
    for i in (0, 7, 23):
        w = ws[i]
        ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, levels[i], w.p, w.sigma)
        tol = 1e-12 if precision == "fp64" else 1e-5
        assert G.rel_l2(res[i][0], res[i][1], ur, vr) <= tol


def test_batch_with_empty_and_tiny_instances():
    _lib = G.lib()
    ws = [W.tiny(n, s, L=3, p=8) for n, s in ((0, 1), (1, 2), (5, 3), (3000, 4))]
    ctx = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
    res = _batch(ctx, ws, [3, 3, 2, 4])
    ctx.close()
    assert res[0][0].size == 0
    assert res[1][0][0] == 0.0
    for w, L, (u, v) in zip(ws[2:], [2, 4], res[2:]):
        ua, va = G.run(w, "mixed", L=L)
        assert np.array_equal(u, ua) and np.array_equal(v, va)


def test_batch_of_512_uneven_instances(orc):
    _lib = G.lib()
    ws = W.batch(n_inst=512, seed=1)
    ctx = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
    res = _batch(ctx, ws, [0] * len(ws))
    ctx.close()
    rng = np.random.default_rng(0)
    for i in rng.choice(512, 6, replace=False):
        w = ws[i]
        L = _lib.petfmm_choose_levels(w.n, w.p, w.sigma, w.domain)
        tg = W.sample_targets(w.n, 256, seed=int(i))
        ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, L, w.p, w.sigma, targets=tg)
        # the mixed path's bar is 1e-5 of the FP64 FMM; the oracle FMM is that FMM
        assert G.rel_l2(res[i][0][tg], res[i][1][tg], ur, vr) <= 1e-5
