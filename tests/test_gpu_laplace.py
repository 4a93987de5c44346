"""The second kernel on the GPU: the 2D logarithmic potential
u_i = sum_{j != i} q_j log|x_i - x_j| (PETFMM_OPT_KERNEL =
PETFMM_KERNEL_LAPLACE), FP64 path, against the oracle's Laplace FMM and
direct sum (pinned in test_oracle_laplace.py).

Bars: the GPU FMM computes the oracle FMM's sums with rescaled (but
mathematically identical) coefficients in another order, so rel-L2 <= 1e-12;
against the direct sum the difference is the FMM's truncation error, which
decays geometrically in p.  The mixed path (FP32 expansions, 3xTF32 tensor-core
M2L, FP32 near field with the SFU logarithm) stays within the vortex kernel's
bar, rel-L2 <= 1e-5 of the FP64 GPU FMM at the same L and p."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def run_laplace(w, L=None, p=None, domain=None, keep=None, precision="fp64", blocks=0):
    _lib = G.lib()
    L = w.L if L is None else L
    p = w.p if p is None else p
    ctx = _lib.Context(domain or w.domain, L, p, w.sigma, precision=precision, dtype=w.dtype,
                       kernel="laplace")
    ctx.set_option(_lib.PETFMM_OPT_POISON, 1)
    ctx.set_option(_lib.PETFMM_OPT_TC_BLOCKS, blocks)
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    u, v = ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    out = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    if keep is not None:
        keep.append(ctx)
    else:
        ctx.close()
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,seed,L,p,frac", [
    (2000, 1, 1, 5, 0.0),      # no far field at all
    (2000, 2, 2, 1, 0.0),      # the log term alone
    (3000, 3, 3, 40, 0.2),     # the largest order
    (5000, 4, 5, 17, 0.5),     # clustered, many empty leaves
    (777, 5, 4, 9, 0.0),       # ragged everything
    (20000, 6, 6, 12, 0.3),
])
def test_laplace_fp64_matches_oracle_fmm(orc, n, seed, L, p, frac):
    w = W.tiny(n, seed, L=L, p=p, clustered_frac=frac)
    ref = orc.laplace_fmm(w.x, w.y, w.gamma, w.domain, L, p)
    u, v = run_laplace(w)
    assert np.all(v == 0.0)
    assert rel(u, ref) <= TOL64


def test_laplace_expansions_match_oracle(orc):
    # ME a~_k = a_k / r^k and LE b^_k = b_k r^k of every occupied box
    w = W.tiny(4000, 11, L=4, p=10, clustered_frac=0.3)
    keep = []
    run_laplace(w, keep=keep)
    ctx = keep[0]
    _, me, le = orc.laplace_fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, export=True)
    _, _, key = orc.bin(w.x, w.y, w.domain, w.L)
    k = np.arange(w.p)
    for level in range(2, w.L + 1):
        r = 1.0 / (1 << level)
        off = ((1 << (2 * level)) - 1) // 3
        nb = 1 << (2 * level)
        occ = np.zeros(nb, bool)
        occ[np.unique(key >> (2 * (w.L - level)))] = True
        me_o = me[off:off + nb][occ] / r ** k
        le_o = le[off:off + nb][occ] * r ** k
        me_g = ctx.debug_expansions(level, 0)[occ]
        le_g = ctx.debug_expansions(level, 1)[occ]
        assert np.max(np.abs(me_g - me_o)) <= 1e-12 * np.max(np.abs(me_o))
        assert np.max(np.abs(le_g - le_o)) <= 1e-12 * np.max(np.abs(le_o))
    ctx.close()


def test_laplace_converges_to_direct_sum(orc):
    w = W.tiny(6000, 21, L=5, p=4, clustered_frac=0.4)
    d = orc.laplace_direct(w.x, w.y, w.gamma)
    errs = [rel(run_laplace(w, p=p)[0], d) for p in (4, 8, 16, 30)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-12


def test_laplace_f32_storage_and_large_sampled(orc):
    # fp32 storage of the inputs and outputs; 200k blobs, sampled targets
    w = W.tiny(200_000, 31, L=7, p=17, clustered_frac=0.3, dtype="f32")
    u, _ = run_laplace(w)
    tg = W.sample_targets(w.n, 300)
    ref = orc.laplace_fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, targets=tg)
    assert rel(u[tg], ref) <= 1e-6   # the output is rounded to FP32 once
    d = orc.laplace_direct(w.x, w.y, w.gamma, targets=tg)
    assert rel(u[tg], d) <= 1e-6


def test_laplace_edge_cases(orc):
    _lib = G.lib()
    torch = G.torch_cuda()
    ctx = _lib.Context((0, 0, 1), 3, 8, 0.01, precision="fp64", dtype="f64", kernel="laplace")
    # one charge: nothing else to feel
    x = torch.tensor([0.3], dtype=torch.float64, device="cuda")
    u, v = ctx.evaluate(x, x.clone(), torch.tensor([2.0], dtype=torch.float64, device="cuda"))
    assert ctx.sync() == 0 and u.item() == 0.0 and v.item() == 0.0
    # coincident charges contribute nothing to each other
    xs = torch.tensor([0.2, 0.2, 0.7], dtype=torch.float64, device="cuda")
    ys = torch.tensor([0.4, 0.4, 0.9], dtype=torch.float64, device="cuda")
    qs = torch.tensor([1.0, -3.0, 0.5], dtype=torch.float64, device="cuda")
    u, v = ctx.evaluate(xs, ys, qs)
    assert ctx.sync() == 0
    # (the third charge is in the far field of the other two at L = 3)
    ref = orc.laplace_fmm(xs.cpu().numpy(), ys.cpu().numpy(), qs.cpu().numpy(), (0, 0, 1), 3, 8)
    assert np.allclose(u.cpu().numpy(), ref, rtol=1e-13, atol=1e-14)
    ctx.close()


def test_vortex_and_laplace_contexts_side_by_side(orc):
    # the kernel is a per-context choice: a vortex context's results do not
    # change when a Laplace context runs in between
    w = W.tiny(5000, 41, L=4, p=12, clustered_frac=0.2)
    u1, v1 = G.run(w, "fp64")
    run_laplace(w)
    u2, v2 = G.run(w, "fp64")
    assert np.array_equal(u1, u2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("case", [
    dict(n=10_000, seed=1, L=4, p=12, frac=0.0),
    dict(n=60_000, seed=2, L=6, p=17, frac=0.5),
    dict(n=300_000, seed=3, L=8, p=17, frac=0.2),   # tensor-core M2L levels
    dict(n=300_000, seed=3, L=8, p=17, frac=0.2, blocks=1),   # ... blocks from level 5
    dict(n=300_000, seed=3, L=8, p=17, frac=0.2, blocks=2),   # ... row units
    dict(n=1000, seed=4, L=2, p=40, frac=0.0),      # no tensor cores at this order
])
def test_laplace_mixed_vs_fp64(case, dtype):
    w = W.tiny(case["n"], case["seed"], L=case["L"], p=case["p"], clustered_frac=case["frac"],
               dtype=dtype)
    u64, _ = run_laplace(w)
    umx, vmx = run_laplace(w, precision="mixed", blocks=case.get("blocks", 0))
    assert np.all(vmx == 0.0)
    assert rel(umx, u64) <= 1e-5


def test_laplace_mixed_against_oracle_sample(orc):
    w = W.laplace_uniform(n=1 << 18, seed=7, L=7, p=17, dtype="f32")
    umx, _ = run_laplace(w, precision="mixed")
    tg = W.sample_targets(w.n, 400)
    ref = orc.laplace_fmm(w.x, w.y, w.gamma, w.domain, w.L, w.p, targets=tg)
    assert rel(umx[tg], ref) <= 1e-5
