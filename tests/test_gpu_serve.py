"""Serving: requests (midpoint-RK2 runs of the vortex method, Sec. 3) admitted
under an HBM budget and batched as they arrive; each result is the same
alone and in the mix, and agrees with an FP64 oracle time-stepper."""
import time

import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _wait(srv, tickets, timeout=300):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout
        time.sleep(0.002)
    return [out[t] for t in tickets]


def _patch(n_side, seed):
    w = W.lattice(side=n_side, seed=seed, L=4, p=8)
    return w.x, w.y, w.gamma, w.sigma


def test_result_same_alone_and_in_mix():
    _lib = G.lib()
    reqs = []
    for i, (side, p, prec) in enumerate([(64, 8, "mixed"), (100, 17, "mixed"), (80, 8, "fp64"),
                                         (120, 17, "mixed"), (50, 8, "fp64")]):
        x, y, g, s = _patch(side, i + 1)
        reqs.append(dict(x=x, y=y, gamma=g, sigma=s, order=p, dt=0.05, n_steps=3, precision=prec))
    alone = []
    for r in reqs:
        srv = _lib.Server(8 << 30, max_slots=8)
        alone.append(_wait(srv, [srv.submit(**r)])[0])
        srv.close()
    srv = _lib.Server(8 << 30, max_slots=8)
    tickets = []
    for r in reqs:  # back to back: the later ones arrive while the first is on the GPU
        tickets.append(srv.submit(**r))
    mixed = _wait(srv, tickets)
    st = srv.stats()
    srv.close()
    for a, m in zip(alone, mixed):
        assert a["status"] == 0 and m["status"] == 0
        assert np.array_equal(a["x"], m["x"]) and np.array_equal(a["y"], m["y"])
        assert m["latency_ms"] >= m["queue_ms"] >= 0.0
        assert a["max_shared"] == 1 and a["rounds"] == 2 * 3
    # the mix really overlapped: requests shared rounds (batched evaluations)
    assert max(m["max_shared"] for m in mixed) >= 2
    assert sum(m["max_shared"] >= 2 for m in mixed) >= 2
    assert st["max_active"] >= 2 and st["completed"] == st["submitted"] == len(reqs)


def test_served_rk2_matches_oracle_stepper(orc):
    _lib = G.lib()
    x, y, g, s = _patch(48, 9)
    dt, steps = 0.05, 2
    srv = _lib.Server(4 << 30)
    res = _wait(srv, [srv.submit(x, y, g, s, 17, dt, steps, precision="fp64")])[0]
    srv.close()
    # reference: the same midpoint-RK2 with the oracle's direct sum (Eq. 9)
    xr, yr = x.copy(), y.copy()
    for _ in range(steps):
        u, v = orc.direct(xr, yr, g, s)
        xh, yh = xr + 0.5 * dt * u, yr + 0.5 * dt * v
        u, v = orc.direct(xh, yh, g, s)
        xr, yr = xr + dt * u, yr + dt * v
    disp = np.sqrt(np.sum((xr - x) ** 2 + (yr - y) ** 2))
    err = np.sqrt(np.sum((res["x"] - xr) ** 2 + (res["y"] - yr) ** 2))
    assert disp > 0 and err < 1e-3 * disp


def test_admission_limits():
    _lib = G.lib()
    x, y, g, s = _patch(32, 1)
    small = _lib.Server(1 << 20)  # 1 MiB: no request fits
    with pytest.raises(_lib.PetfmmError) as e:
        small.submit(x, y, g, s, 8, 0.05, 1)
    assert e.value.code == _lib.PETFMM_ENOMEM
    small.close()
    srv = _lib.Server(4 << 30, max_slots=1, max_queue=2)
    ts = [srv.submit(x, y, g, s, 8, 0.05, 2)]
    got_busy = False
    for _ in range(8):
        try:
            ts.append(srv.submit(x, y, g, s, 8, 0.05, 2))
        except _lib.PetfmmError as err:
            assert err.code == _lib.PETFMM_EBUSY
            got_busy = True
            break
    res = _wait(srv, ts)
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert got_busy or len(ts) == 9


def test_release_while_worker_runs():
    # a finished request belongs to the caller: polling (which releases it)
    # as fast as possible while new requests arrive and the worker keeps
    # running rounds must never let the worker touch a released request
    _lib = G.lib()
    srv = _lib.Server(8 << 30, max_slots=16, max_queue=4096)
    rng = np.random.default_rng(3)
    pending, results = [], []
    for i in range(300):
        x, y, g, s = _patch(int(rng.integers(4, 24)), i)
        pending.append(srv.submit(x, y, g, s, 8, 0.05, int(rng.integers(1, 3))))
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                results.append(r)
                pending.remove(t)
    results += _wait(srv, pending)
    srv.close()
    assert len(results) == 300 and all(r["status"] == 0 for r in results)
