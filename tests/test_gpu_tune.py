"""The batch autotuner on the GPU: it returns one rule per (order, N-bucket)
class, installs rules and options in the context, the tuned batch still
matches the oracle FMM per instance (at each instance's tuned L), and a
second run is served from the JSON cache with identical results."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import tuning
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _insts(ws):
    torch = G.torch_cuda()
    out = []
    for w in ws:
        x, y, g = G.to_dev((w.x, w.y, w.gamma))
        out.append(dict(domain=w.domain, levels=0, order=w.p, sigma=w.sigma, x=x, y=y, gamma=g,
                        u=torch.empty_like(x), v=torch.empty_like(x)))
    return out


def test_tuned_batch_matches_oracle_per_instance(orc, tmp_path):
    _lib = G.lib()
    torch = G.torch_cuda()
    ws = W.batch(n_inst=40, seed=9, n_min=1000, n_max=60_000)
    insts = _insts(ws)
    ctx = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
    ctx.set_option(_lib.PETFMM_OPT_GRAPH, 1)
    rules, rep = ctx.tune_batch(insts, reps=2)
    classes = tuning.batch_classes([dict(order=w.p, n=w.n) for w in ws])
    assert rep["nrules"] == len(rules) == len(classes)
    assert {f"{r['order']}:{r['log2n']}" for r in rules} == classes
    assert rep["ms_tuned"] > 0 and rep["ms_model"] > 0 and rep["evaluations"] > len(rules)
    assert rep["tc_blocks"] in (0, 1, 2) and rep["tc_dense_pct"] in (1, 5)
    # the tuned batch through the public entry point (levels <= 0: the rules)
    ctx.evaluate_batch(insts)
    assert ctx.sync() == 0
    res = [(it["u"].cpu().numpy(), it["v"].cpu().numpy()) for it in insts]
    ctx.close()
    for i in (0, 9, 17, 26, 39):
        w = ws[i]
        L = _lib.petfmm_rule_levels(rules, w.n, w.p, w.sigma, w.domain)
        tg = W.sample_targets(w.n, 256, seed=i)
        ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, L, w.p, w.sigma, targets=tg)
        assert G.rel_l2(res[i][0][tg], res[i][1][tg], ur, vr) <= 1e-5
    # the cache: a tuner run is saved, the next call is a hit with the same
    # rules and options, and the batch gives the same bits
    path = str(tmp_path / "tune.json")
    dev = tuning.device_key(torch.cuda.get_device_name(), torch.cuda.get_device_properties(0).multi_processor_count)
    ctx1 = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
    s1 = tuning.autotune(ctx1, insts, path, dev, reps=1)
    assert not s1["from_cache"]
    ctx1.evaluate_batch(insts)
    assert ctx1.sync() == 0
    a = [it["u"].cpu().numpy().copy() for it in insts]
    ctx1.close()
    ctx2 = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
    s2 = tuning.autotune(ctx2, insts, path, dev)
    assert s2["from_cache"] and s2["options"] == s1["options"]
    assert sorted((r["order"], r["log2n"], r["levels"]) for r in s2["rules"]) == \
        sorted((r["order"], r["log2n"], r["levels"]) for r in s1["rules"])
    ctx2.evaluate_batch(insts)
    assert ctx2.sync() == 0
    b = [it["u"].cpu().numpy() for it in insts]
    ctx2.close()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
