"""The autotuner's host logic (no GPU): the level-rule lookup the batched
evaluation applies (petfmm_rule_levels, through the C ABI) and the JSON cache
keyed by (device, p, N-bucket)."""
import json
import math

import pytest

import __graft_entry__
from paper_0905_2637_gb300 import tuning


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


DOM = (0.0, 0.0, 1.0)


def test_rule_levels_follow_rules_else_the_work_model(lib):
    n, p = 50_000, 17
    sigma = 0.5 / math.sqrt(n)
    model = lib.petfmm_choose_levels(n, p, sigma, DOM)
    e = n.bit_length() - 1
    # no rules: the model
    assert lib.petfmm_rule_levels([], n, p, sigma, DOM) == model
    # a matching rule wins when the guard allows it
    lower = max(1, model - 1)
    assert lib.petfmm_rule_levels([dict(order=p, log2n=e, levels=lower)], n, p, sigma, DOM) == lower
    # rules for another order or bucket are ignored
    other = [dict(order=12, log2n=e, levels=lower), dict(order=p, log2n=e + 1, levels=lower)]
    assert lib.petfmm_rule_levels(other, n, p, sigma, DOM) == model
    # a rule the kernel-substitution guard forbids (leaves narrower than
    # sigma sqrt(2 ln 1e8)) falls back to the model
    rmin = sigma * math.sqrt(2 * math.log(1e8))
    too_deep = next(L for L in range(1, 16) if 1.0 / 2 ** L < rmin)
    assert lib.petfmm_rule_levels([dict(order=p, log2n=e, levels=too_deep)], n, p, sigma, DOM) == model


def test_rule_levels_bucket_is_floor_log2(lib):
    sigma = 1e-4
    rules = [dict(order=8, log2n=10, levels=3)]
    assert lib.petfmm_rule_levels(rules, 1024, 8, sigma, DOM) == 3   # 2^10
    assert lib.petfmm_rule_levels(rules, 2047, 8, sigma, DOM) == 3   # still bucket 10
    m = lib.petfmm_choose_levels(2048, 8, sigma, DOM)
    assert lib.petfmm_rule_levels(rules, 2048, 8, sigma, DOM) == m    # bucket 11


def test_bucket_and_class_keys():
    assert tuning.log2_bucket(1) == 0
    assert tuning.log2_bucket(1023) == 9 and tuning.log2_bucket(1024) == 10
    with pytest.raises(ValueError):
        tuning.log2_bucket(0)
    insts = [dict(order=8, n=1000), dict(order=8, n=1023), dict(order=17, n=4096), dict(order=12, n=0)]
    assert tuning.batch_classes(insts) == {"8:9", "17:12"}


def test_cache_round_trip_merge_and_coverage(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    dev = tuning.device_key("NVIDIA GB300", 152)
    c = tuning.TuningCache(path)                      # missing file: empty
    assert c.lookup(dev, {"8:9"}) is None
    c.update(dev, [dict(order=8, log2n=9, levels=3, ms=0.2), dict(order=17, log2n=12, levels=4, ms=0.5)],
             dict(tc_blocks=1, tc_dense_pct=5))
    c.save()
    d = tuning.TuningCache(path)
    rules, opts = d.lookup(dev, {"8:9", "17:12"})
    assert opts == {"tc_blocks": 1, "tc_dense_pct": 5}
    assert [(r["order"], r["log2n"], r["levels"]) for r in rules] == [(17, 12, 4), (8, 9, 3)]
    assert d.lookup(dev, {"8:9", "12:10"}) is None    # a class not tuned yet
    assert d.lookup("other/1", {"8:9"}) is None       # another device
    # a later run replaces its classes only, and the options
    d.update(dev, [dict(order=8, log2n=9, levels=4, ms=0.1)], dict(tc_blocks=0, tc_dense_pct=1))
    d.save()
    e = tuning.TuningCache(path)
    rules, opts = e.lookup(dev, {"8:9", "17:12"})
    assert {(r["order"], r["levels"]) for r in rules} == {(8, 4), (17, 4)}
    assert opts == {"tc_blocks": 0, "tc_dense_pct": 1}
    assert json.load(open(path))["version"] == tuning.VERSION


def test_cache_ignores_a_corrupt_file(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    c = tuning.TuningCache(str(path))
    assert c.data["devices"] == {}
    path.write_text(json.dumps({"version": 999, "devices": {"x": {}}}))
    assert tuning.TuningCache(str(path)).data["devices"] == {}


def test_summary_counts_changes_against_the_model():
    rules = [dict(order=8, log2n=9, levels=3, ms=1.0), dict(order=17, log2n=12, levels=5, ms=3.0)]
    s = tuning.summarize(rules, {"8:9": 3, "17:12": 4})
    assert s["classes"] == 2 and s["changed_vs_model"] == 1 and s["levels"] == [3, 5]
    assert s["mean_ms"] == 2.0


def test_set_level_rules_rejects_bad_rules_without_a_gpu(lib):
    import ctypes
    # a null context is rejected before anything else
    arr = (lib.LevelRule * 1)(lib.LevelRule(8, 9, 3, 0.0))
    assert lib.load().petfmm_set_level_rules(None, arr, 1) == lib.PETFMM_EINVAL
    rep = lib.TuneReport()
    assert lib.load().petfmm_tune_batch(None, 0, None, 1, None, 0, ctypes.byref(rep)) == lib.PETFMM_EINVAL
