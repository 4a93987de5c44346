"""The bounds-checked build (libpetfmm_checked.so, -DPETFMM_CHECKS) on small
cases that reach every checked path: directed and pairwise near field, split
heavy pairs, the FP64 path, a batch with empty instances, and the Laplace
kernel.  Every index read from device data must pass its check (no recorded
failure), and the results must still match the oracle FMM.  Runs in a child
process, which loads the checked library instead of the regular one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle
from paper_0905_2637_gb300 import _lib
from paper_0905_2637_gb300 import workloads as W
assert _lib.LIB_PATH.endswith("libpetfmm_checked.so")
oracle.build()
lines = (__import__("ctypes").c_uint32 * 3)()

def clean(what):
    n = _lib.load().petfmm_debug_checks(lines)
    assert n == 3, n
    assert list(lines) == [0, 0, 0], (what, list(lines))

def rel(u, v, ur, vr):
    return float(np.sqrt(np.sum((u - ur) ** 2 + (v - vr) ** 2) / np.sum(ur ** 2 + vr ** 2)))

cases = [
    ("mixed pairs", W.tiny(20_000, 1, L=4, p=12, clustered_frac=0.4), "mixed", {}, 1e-5),
    ("split pairs", W.tiny(40_000, 2, L=2, p=8, clustered_frac=0.6), "mixed", {}, 1e-5),
    ("directed", W.tiny(20_000, 3, L=4, p=12), "mixed", {_lib.PETFMM_OPT_P2P_PAIRS: 0}, 1e-5),
    ("fp64", W.tiny(8_000, 4, L=4, p=10, clustered_frac=0.3), "fp64", {}, 1e-12),
]
for what, w, prec, opts, tol in cases:
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision=prec, dtype=w.dtype)
    for k, v in opts.items():
        ctx.set_option(k, v)
    x, y, g = (torch.from_numpy(a).cuda() for a in (w.x, w.y, w.gamma))
    u, v = ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    u, v = u.cpu().numpy(), v.cpu().numpy()
    ctx.close()
    clean(what)
    ur, vr = oracle.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    e = rel(u, v, ur, vr)
    assert e <= tol, (what, e)
    print(what, "ok", e)
# a batch with empty and tiny instances
ws = [W.tiny(n, s, L=3, p=8) for n, s in ((0, 11), (1, 12), (700, 13), (5000, 14))]
ctx = _lib.Context((0, 0, 1), 2, 8, 0.01, precision="mixed", dtype="f64")
insts = []
for w in ws:
    x, y, g = (torch.from_numpy(a).cuda() for a in (w.x, w.y, w.gamma))
    insts.append(dict(domain=w.domain, levels=0, order=w.p, sigma=w.sigma, x=x, y=y, gamma=g,
                      u=torch.empty_like(x), v=torch.empty_like(x)))
ctx.evaluate_batch(insts)
assert ctx.sync() == 0
ctx.close()
clean("batch")
# the Laplace kernel
w = W.tiny(10_000, 15, L=4, p=12)
ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype="f64", kernel="laplace")
x, y, g = (torch.from_numpy(a).cuda() for a in (w.x, w.y, w.gamma))
u, v = ctx.evaluate(x, y, g)
assert ctx.sync() == 0
ctx.close()
clean("laplace")
print("CHECKED-OK")
'''


def test_checked_build_reports_no_out_of_range_index():
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ, PETFMM_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "CHECKED-OK" in r.stdout
