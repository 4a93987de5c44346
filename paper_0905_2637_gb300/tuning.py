"""Persistent cache of the batch autotuner's results (``petfmm_tune_batch``).

The tuner times candidate tree depths per class of instances -- same order p,
same floor(log2 N) -- and the M2L shape options for a batch, on the GPU.  Its
winners depend on the device, so the cache is keyed by (device, p, N-bucket)
for the level rules and by device for the options, and stored as JSON:

    {"version": 1,
     "devices": {"NVIDIA GB300/152": {
         "rules": {"17:14": {"levels": 9, "ms": 0.41}, ...},
         "options": {"tc_blocks": 0, "tc_dense_pct": 1}}}}

``autotune`` installs cached results in a context when they cover every class
of the batch, and otherwise runs the tuner and merges what it found.  This
module does no arithmetic of the method; it only files and looks up results.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

VERSION = 1


def log2_bucket(n: int) -> int:
    """floor(log2 n), the N-bucket of a class (n >= 1)."""
    if n < 1:
        raise ValueError("a class needs at least one particle")
    return int(n).bit_length() - 1


def class_key(order: int, n: int) -> str:
    return f"{int(order)}:{log2_bucket(n)}"


def batch_classes(instances) -> set:
    """The (order, N-bucket) keys of a batch's non-empty instances."""
    out = set()
    for it in instances:
        n = int(it["n"]) if "n" in it else int(it["x"].numel())
        if n > 0:
            out.add(class_key(it["order"], n))
    return out


def device_key(name: str, sms: int) -> str:
    return f"{name}/{int(sms)}"


class TuningCache:
    """The JSON file of tuned results (missing or unreadable file: empty)."""

    def __init__(self, path: str):
        self.path = path
        self.data = {"version": VERSION, "devices": {}}
        try:
            with open(path) as f:
                d = json.load(f)
            if isinstance(d, dict) and d.get("version") == VERSION and isinstance(d.get("devices"), dict):
                self.data = d
        except (OSError, ValueError):
            pass

    def _dev(self, dev: str) -> dict:
        return self.data["devices"].setdefault(dev, {"rules": {}, "options": None})

    def lookup(self, dev: str, classes) -> tuple | None:
        """(rules, options) covering every class, or None if any is missing."""
        d = self.data["devices"].get(dev)
        if not d or not d.get("options"):
            return None
        rules = []
        for key in sorted(classes):
            r = d["rules"].get(key)
            if r is None:
                return None
            p, e = (int(v) for v in key.split(":"))
            rules.append({"order": p, "log2n": e, "levels": int(r["levels"]),
                          "ms": float(r.get("ms", 0.0))})
        return rules, dict(d["options"])

    def update(self, dev: str, rules, options: dict) -> None:
        """Merge a tuner run: its rules replace those of the same classes; the
        options replace the device's."""
        d = self._dev(dev)
        for r in rules:
            d["rules"][f"{int(r['order'])}:{int(r['log2n'])}"] = {
                "levels": int(r["levels"]), "ms": float(r.get("ms", 0.0))}
        d["options"] = {"tc_blocks": int(options["tc_blocks"]),
                        "tc_dense_pct": int(options["tc_dense_pct"])}

    def save(self) -> None:
        """Write atomically (a temporary file in the same folder, renamed)."""
        folder = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(folder, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tuning", dir=folder)
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune(ctx, instances, cache_path: str, device: str, reps: int = 3) -> dict:
    """Install tuned rules and options in ctx for this batch: from the cache
    when it covers the batch's classes, else by running the tuner on the GPU
    (which leaves the tuned batch's result in the instances' u, v) and saving
    the winners.  Returns a summary dict."""
    from . import _lib
    cache = TuningCache(cache_path)
    classes = batch_classes(instances)
    hit = cache.lookup(device, classes)
    if hit is not None:
        rules, opts = hit
        ctx.set_level_rules(rules)
        ctx.set_option(_lib.PETFMM_OPT_TC_BLOCKS, opts["tc_blocks"])
        ctx.set_option(_lib.PETFMM_OPT_TC_DENSE, opts["tc_dense_pct"])
        return {"from_cache": True, "rules": rules, "options": opts, "report": None}
    rules, rep = ctx.tune_batch(instances, reps=reps)
    opts = {"tc_blocks": rep["tc_blocks"], "tc_dense_pct": rep["tc_dense_pct"]}
    cache.update(device, rules, opts)
    cache.save()
    return {"from_cache": False, "rules": rules, "options": opts, "report": rep}


def summarize(rules, model_levels: dict | None = None) -> dict:
    """Counts for a report: classes, and how many tuned depths differ from
    the work model's (model_levels: class key -> model L)."""
    changed = None
    if model_levels is not None:
        changed = sum(1 for r in rules
                      if model_levels.get(f"{r['order']}:{r['log2n']}") not in (None, r["levels"]))
    return {"classes": len(rules), "changed_vs_model": changed,
            "levels": sorted({int(r["levels"]) for r in rules}) if rules else [],
            "mean_ms": (sum(r.get("ms", 0.0) for r in rules) / len(rules)) if rules else math.nan}
