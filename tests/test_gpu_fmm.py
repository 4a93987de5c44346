"""End-to-end parity of the CUDA FMM with the FP64 oracle.

Bars (written here, derived from the arithmetic): the FP64 GPU FMM computes
the oracle's sums with rescaled (but mathematically identical) expansion
coefficients and another summation order, so it agrees to rounding:
rel-L2 <= 1e-12.  The mixed path (FP32 expansions and near field, rescaled
operators rounded to FP32) must stay within rel-L2 <= 1e-5 of the FP64 FMM at
the same L and p."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMX = 1e-5


def test_uniform_10k_fp64_all_targets(orc):
    w = W.uniform()
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    u, v = G.run(w, "fp64")
    assert G.rel_l2(u, v, ur, vr) <= TOL64
    # and against the direct sum of Eq. 9 the error is the truncation error
    ud, vd = orc.direct(w.x, w.y, w.gamma, w.sigma)
    assert G.rel_l2(u, v, ud, vd) < 1e-3


@pytest.mark.parametrize("n,seed,L,p,frac", [
    (2000, 1, 1, 5, 0.0),      # no far field at all
    (2000, 2, 2, 1, 0.0),      # a single expansion term
    (3000, 3, 3, 40, 0.2),     # the largest order
    (5000, 4, 5, 17, 0.5),     # clustered, many empty leaves
    (777, 5, 4, 9, 0.0),       # ragged everything
    (20000, 6, 6, 12, 0.3),
])
def test_fp64_sweep(orc, n, seed, L, p, frac):
    w = W.tiny(n, seed, L=L, p=p, clustered_frac=frac)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, L, p, w.sigma)
    u, v = G.run(w, "fp64")
    assert G.rel_l2(u, v, ur, vr) <= TOL64


def test_fp64_expansions_match_oracle(orc):
    # Verification dump of Sec. 6.2: ME and LE of every box, compared in the
    # scaled form (ME a_k / r^k, LE r^(k+1) b_k).
    w = W.tiny(4000, 11, L=4, p=10, clustered_frac=0.3)
    _lib = G.lib()
    keep = []
    G.run(w, "fp64", ctx_out=keep)
    ctx = keep[0]
    _, _, me, le = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, export=True)
    _, _, key = orc.bin(w.x, w.y, w.domain, w.L)
    k = np.arange(w.p)
    for level in range(2, w.L + 1):
        r = 1.0 / (1 << level)
        off = ((1 << (2 * level)) - 1) // 3
        nb = 1 << (2 * level)
        # boxes holding particles (empty boxes are skipped by the library: their
        # ME is zero and their LE is never evaluated)
        occ = np.zeros(nb, bool)
        occ[np.unique(key >> (2 * (w.L - level)))] = True
        me_o = me[off:off + nb][occ] / r ** k
        le_o = le[off:off + nb][occ] * r ** (k + 1)
        me_g = ctx.debug_expansions(level, 0)[occ]
        le_g = ctx.debug_expansions(level, 1)[occ]
        assert np.max(np.abs(me_g - me_o)) <= 1e-12 * np.max(np.abs(me_o))
        assert np.max(np.abs(le_g - le_o)) <= 1e-12 * np.max(np.abs(le_o))
        assert np.all(me[off:off + nb][~occ] == 0)
    ctx.close()


def test_lattice_1m_fp64_and_mixed(orc):
    w = W.lattice()
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    u64, v64 = G.run(w, "fp64")
    assert G.rel_l2(u64, v64, ur, vr) <= TOL64
    umx, vmx = G.run(w, "mixed")
    assert G.rel_l2(umx, vmx, u64, v64) <= TOLMX
    # 4096 seeded targets against the direct sum (O1): the kernel-substitution
    # (Type I) floor is a few 1e-6 here, so a bar of 1e-5 catches a near-field
    # regression that the FMM-against-FMM checks would not see
    tg = W.sample_targets(w.n, 4096)
    ud, vd = orc.direct(w.x, w.y, w.gamma, w.sigma, targets=tg)
    assert G.rel_l2(u64[tg], v64[tg], ud, vd) <= 1e-5
    assert G.rel_l2(umx[tg], vmx[tg], ud, vd) <= 1e-5


def test_clustered_16m_mixed_vs_fp64_and_oracle_sample(orc):
    w = W.clustered()
    # the FP64 path on FP64 copies of the same (FP32-valued) inputs, so that
    # its outputs are not rounded to FP32 storage
    w64 = W.Workload(w.name, *w.as_f64(), w.sigma, w.domain, w.L, w.p, "f64")
    u64, v64 = G.run(w64, "fp64")
    umx, vmx = G.run(w, "mixed")
    assert G.rel_l2(umx, vmx, u64, v64) <= TOLMX
    tg = W.sample_targets(w.n, 4096, seed=3)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, targets=tg)
    assert G.rel_l2(u64[tg], v64[tg], ur, vr) <= TOL64


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("case", [
    dict(n=10_000, seed=1, L=4, p=12, frac=0.0),
    dict(n=30_000, seed=2, L=6, p=17, frac=0.5),
    dict(n=1000, seed=3, L=2, p=40, frac=0.0),
])
def test_mixed_vs_fp64_sweep(case, dtype):
    w = W.tiny(case["n"], case["seed"], L=case["L"], p=case["p"], clustered_frac=case["frac"], dtype=dtype)
    u64, v64 = G.run(w, "fp64")
    umx, vmx = G.run(w, "mixed")
    assert G.rel_l2(umx, vmx, u64, v64) <= TOLMX


def test_mixed_general_near_field_branch(orc):
    # sigma small against the leaf: the near field reaches q >> 1, so the
    # kernel takes the exp/division branch above the polynomial range
    w = W.tiny(20_000, 9, L=4, p=12, sigma=0.003)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    umx, vmx = G.run(w, "mixed")
    assert G.rel_l2(umx, vmx, ur, vr) <= TOLMX


def test_empty_and_single_particle():
    _lib = G.lib()
    torch = G.torch_cuda()
    for precision in ("fp64", "mixed"):
        ctx = _lib.Context((0, 0, 1), 3, 8, 0.01, precision=precision, dtype="f64")
        e = torch.empty(0, dtype=torch.float64, device="cuda")
        ctx.evaluate(e, e, e, e.clone(), e.clone())
        assert ctx.sync() == 0
        x, y, g = G.to_dev((np.array([0.3]), np.array([0.7]), np.array([2.0])))
        u, v = ctx.evaluate(x, y, g)
        assert ctx.sync() == 0
        assert u.item() == 0.0 and v.item() == 0.0
        ctx.close()


def test_coincident_particles_and_self_are_zero(orc):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 500)
    y = rng.uniform(0, 1, 500)
    x[100:110] = x[99]
    y[100:110] = y[99]
    w = W.Workload("coincident", x, y, rng.uniform(-1, 1, 500), 0.02, (0, 0, 1), 3, 10, "f64")
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma)
    u, v = G.run(w, "fp64")
    assert G.rel_l2(u, v, ur, vr) <= TOL64
    umx, vmx = G.run(w, "mixed")
    assert np.all(np.isfinite(umx)) and G.rel_l2(umx, vmx, u, v) <= TOLMX


def test_near_field_tolerance_option():
    # The near-field factor's polynomial is fitted to the context's tolerance
    # (default 2.5e-6): both it and the FP32-rounding-level fit (1e-7) keep
    # the mixed path within the 1e-5 bar; out-of-range values are rejected.
    _lib = G.lib()
    w = W.tiny(40_000, 12, L=6, p=17, clustered_frac=0.6, dtype="f32")
    u64, v64 = G.run(w, "fp64")
    errs = {}
    for tol in (None, 100, 2500, 20000):
        opts = {} if tol is None else {_lib.PETFMM_OPT_NEAR_TOL: tol}
        umx, vmx = G.run(w, "mixed", options=opts)
        errs[tol] = G.rel_l2(umx, vmx, u64, v64)
    assert errs[None] == errs[2500]              # the default is 2.5e-6
    assert errs[100] <= TOLMX and errs[2500] <= TOLMX
    assert errs[20000] < 5e-5                   # a loose fit: loose, bounded result
    ctx = _lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype=w.dtype)
    for bad in (0, -5, 1_000_001):
        with pytest.raises(_lib.PetfmmError):
            ctx.set_option(_lib.PETFMM_OPT_NEAR_TOL, bad)
    ctx.close()


def test_lamb_oseen_paper_case(orc):
    # Sec. 7.1 at the paper's size: 875^2 lattice blobs, sigma = 0.02,
    # h = 0.8 sigma, L = 10, p = 17 (leaves narrower than the lattice
    # spacing: about one blob per occupied leaf, M2L-dominated)
    w = W.lamb_oseen_paper(dtype="f64")  # FP64 outputs for the 1e-12 comparison
    assert w.n == 875 * 875
    u64, v64 = G.run(w, "fp64")
    umx, vmx = G.run(w, "mixed")
    assert G.rel_l2(umx, vmx, u64, v64) <= TOLMX
    tg = W.sample_targets(w.n, 512, seed=11)
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, w.sigma, targets=tg)
    assert G.rel_l2(u64[tg], v64[tg], ur, vr) <= TOL64
