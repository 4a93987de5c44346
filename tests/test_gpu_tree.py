"""Morton binning, radix sort and leaf ranges on the GPU are bit-exact
against the oracle (Sec. 2.1 binning, z-order of Sec. 5.1, stable order)."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tree(w, precision="mixed", opts=()):
    _lib = G.lib()
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision=precision, dtype=w.dtype)
    for k, v in opts:
        ctx.set_option(getattr(_lib, k), v)
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    keys, perm, start = ctx.debug_tree(w.n)
    ctx.close()
    return keys, perm, start


def _check(orc, w, precision="mixed", opts=()):
    xd, yd, _ = w.as_f64()
    _, _, key = orc.bin(xd, yd, w.domain, w.L)
    perm, start = orc.sort(key, w.L)
    k2, p2, s2 = _tree(w, precision, opts)
    assert np.array_equal(k2, key)
    assert np.array_equal(p2, perm)
    assert np.array_equal(s2, start)


@pytest.mark.parametrize("case", [
    dict(n=10_000, seed=1, L=4),                      # uniform, ~39 per leaf
    dict(n=4_097, seed=2, L=3, clustered_frac=0.5),   # ragged tiles, one hot leaf
    dict(n=1, seed=3, L=2),
    dict(n=300_000, seed=4, L=7, clustered_frac=0.3),  # several sort tiles, 2 radix passes
    dict(n=50_000, seed=5, L=12),                     # 24-bit keys, 3 passes, mostly empty leaves
])
def test_tree_matches_oracle(orc, case):
    w = W.tiny(case["n"], case["seed"], L=case["L"], clustered_frac=case.get("clustered_frac", 0.0))
    _check(orc, w)


def test_tree_fp64_path_and_f32_storage(orc):
    _check(orc, W.tiny(20_000, 6, L=5), precision="fp64")
    _check(orc, W.tiny(20_000, 7, L=6, dtype="f32"), precision="mixed")


def test_tree_boundaries_and_shifted_domain(orc):
    # points on the domain edges and on box boundaries; a shifted, non-unit domain
    dom = (-2.0, 3.0, 4.0)
    L = 5
    edges = np.array([-2.0, 2.0, 0.0, -2.0 + 4.0 / 32, np.nextafter(-2.0 + 4.0 / 32, -3.0)])
    rng = np.random.default_rng(0)
    x = np.concatenate([edges, rng.uniform(-2, 2, 995)])
    y = np.concatenate([np.array([3.0, 7.0, 5.0, 7.0, 3.0]), rng.uniform(3, 7, 995)])
    w = W.Workload("edges", x, y, rng.uniform(-1, 1, 1000), 0.01, dom, L, 8, "f64")
    _check(orc, w)


def test_tree_all_particles_in_one_leaf(orc):
    rng = np.random.default_rng(1)
    x = 0.51 + 1e-4 * rng.uniform(size=5000)
    y = 0.26 + 1e-4 * rng.uniform(size=5000)
    w = W.Workload("one-leaf", x, y, rng.uniform(-1, 1, 5000), 0.01, (0, 0, 1), 6, 8, "f64")
    _check(orc, w)


def test_tree_full_lattice_and_clustered(orc):
    _check(orc, W.lattice())
    _check(orc, W.clustered())


def test_lattice_has_sixteen_per_leaf():
    w = W.lattice()
    _, _, start = _tree(w)
    assert np.all(np.diff(start) == 16)


def test_outside_particle_reports_edomain_then_recovers():
    _lib = G.lib()
    w = W.tiny(1000, 8, L=3)
    x = w.x.copy()
    x[17] = 1.0 + 1e-9
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype="f64")
    xd, yd, gd = G.to_dev((x, w.y, w.gamma))
    ctx.evaluate(xd, yd, gd)
    with pytest.raises(_lib.PetfmmError) as e:
        ctx.sync()
    assert e.value.code == _lib.PETFMM_EDOMAIN
    xd, yd, gd = G.to_dev((w.x, w.y, w.gamma))
    ctx.evaluate(xd, yd, gd)
    assert ctx.sync() == 0
    xn = w.x.copy()
    xn[3] = np.nan
    xd = G.to_dev((xn,))[0]
    ctx.evaluate(xd, yd, gd)
    with pytest.raises(_lib.PetfmmError) as e:
        ctx.sync()
    assert e.value.code == _lib.PETFMM_EDOMAIN
    ctx.close()


@pytest.mark.parametrize("L", [10, 3])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("dom", [(0.1234567891, -0.3718281828, 0.7071067811865476),
                                 (1.0e5 + 0.3, -2.5e4, 3.0), (-2.0, 1.0, 4.0)])
def test_binning_near_bin_edges(orc, dtype, dom, L):
    # The kernel bins in FP32 where that provably gives the FP64 bin and falls
    # back to FP64 otherwise: points on and a few ulps around every bin edge
    # of one row -- the domain's own edges included -- in awkward domains (x0
    # and the scale not representable in FP32; one so far from the origin that
    # FP32 never decides; one straddling it), on a deep and a shallow tree
    nb = 1 << L
    x0, y0, wd = dom
    ft = np.float32 if dtype == "f32" else np.float64
    e = (x0 + np.arange(nb + 1) * (wd / nb)).astype(ft)
    x = [e]
    for direction in (np.inf, -np.inf):
        v = e
        for _ in range(3):
            v = np.nextafter(v, ft(direction))
            x.append(v)
    x = np.concatenate(x)
    xd = x.astype(np.float64)
    x = x[(xd >= x0) & (xd <= x0 + wd)]
    rng = np.random.default_rng(11)
    y = (y0 + rng.uniform(0.01 * wd, 0.99 * wd, x.size)).astype(ft)
    g = rng.uniform(-1, 1, x.size).astype(ft)
    w = W.Workload("bin-edges", x, y, g, 0.01, dom, L, 8, dtype)
    _check(orc, w)
