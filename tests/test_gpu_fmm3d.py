"""The 3D extension on the GPU (the octree FMM of the Laplace potential and
field, fmm3d.cu) against the 3D oracle: tree bit-exact, the FP64 path within
1e-12 of the oracle's FMM, the mixed path within its FP32 budget of the FP64
path, plus the edge cases (one leaf level, empty input, a particle outside
the cube, coincident particles)."""
import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(w, precision):
    from paper_0905_2637_gb300 import fmm3d
    G.lib()
    return fmm3d.Context3D(w.domain, w.L, w.p, precision=precision, dtype=w.dtype)


def _run(w, precision, ctx=None):
    own = ctx is None
    ctx = ctx or _ctx(w, precision)
    args = G.to_dev((w.x, w.y, w.z, w.q))
    out = ctx.evaluate(*args)
    rc = ctx.sync()
    res = tuple(t.cpu().numpy().astype(np.float64) for t in out)
    if own:
        ctx.close()
    return rc, res


def _rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def _field_rel(a, b):
    return float(np.sqrt(sum(np.sum((u - v) ** 2) for u, v in zip(a[1:], b[1:])) /
                         sum(np.sum(v ** 2) for v in b[1:])))


@pytest.mark.parametrize("case", [
    dict(n=5000, seed=1, L=3),
    dict(n=4097, seed=2, L=4, clustered_frac=0.6),
    dict(n=1, seed=3, L=2),
    dict(n=300_000, seed=4, L=6, clustered_frac=0.3),   # 18-bit keys: 3 radix passes
])
def test_tree_matches_oracle(orc, case):
    w = W.tiny3d(case["n"], case["seed"], L=case["L"],
                 clustered_frac=case.get("clustered_frac", 0.0))
    w.x[0], w.y[0], w.z[0] = 1.0, 0.0, 1.0              # corner of the closed cube
    ctx = _ctx(w, "mixed")
    rc, _ = _run(w, "mixed", ctx)
    assert rc == 0
    skeys, perm, start = ctx.debug_tree(w.n)
    ctx.close()
    key = orc.bin3d(w.x, w.y, w.z, w.domain, w.L)
    operm, ostart = orc.sort3d(key, w.L)
    assert np.array_equal(perm, operm)
    assert np.array_equal(skeys, key[operm])
    assert np.array_equal(start, ostart)


@pytest.mark.parametrize("case", [
    dict(n=3000, seed=5, L=2, p=6),
    dict(n=8000, seed=6, L=3, p=8, clustered_frac=0.5),
    dict(n=2000, seed=7, L=1, p=4),          # no far field: the direct sum
    dict(n=6000, seed=8, L=4, p=10, clustered_frac=0.3),
    dict(n=5000, seed=9, L=3, p=16),         # the largest order
])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fp64_path_matches_oracle_fmm(orc, case, dtype):
    w = W.tiny3d(case["n"], case["seed"], L=case["L"], p=case["p"], dtype=dtype,
                 clustered_frac=case.get("clustered_frac", 0.0))
    rc, got = _run(w, "fp64")
    assert rc == 0
    ref = orc.fmm3d(*w.as_f64(), w.domain, w.L, w.p)
    # FP32 storage rounds each output once (relative 2^-24; a 1e-12 difference
    # before it can move the rounding by one ulp, 2^-23)
    tol = 1e-12 if dtype == "f64" else 2.0 ** -23
    assert _rel(got[0], ref[0]) <= tol
    assert _field_rel(got, ref) <= tol


@pytest.mark.parametrize("case", [
    dict(n=20000, seed=10, L=3, p=8),
    dict(n=30000, seed=11, L=4, p=12, clustered_frac=0.5),
    dict(n=20000, seed=12, L=4, p=16, clustered_frac=0.2),
    # small orders: real M2M / L2L with partly filled lanes, odd coefficient
    # counts in the pipelined M2L's row copies (p = 5: 15 complex)
    dict(n=15000, seed=21, L=3, p=3),
    dict(n=20000, seed=22, L=4, p=5, clustered_frac=0.4),
    dict(n=40000, seed=23, L=5, p=7, clustered_frac=0.3),
])
def test_mixed_path_within_fp32_budget_of_fp64(orc, case):
    # FP32 arithmetic (relative rounding 6e-8 per operation) over sums of a
    # few thousand terms and the M2L / L2P series: the budget is 1e-5 relative
    # L2, the bar of the 2D mixed path
    w = W.tiny3d(case["n"], case["seed"], L=case["L"], p=case["p"], dtype="f32",
                 clustered_frac=case.get("clustered_frac", 0.0))
    rc, mixed = _run(w, "mixed")
    assert rc == 0
    rc, fp64 = _run(w, "fp64")
    assert rc == 0
    assert _rel(mixed[0], fp64[0]) <= 1e-5
    assert _field_rel(mixed, fp64) <= 1e-5
    ref = orc.fmm3d(*w.as_f64(), w.domain, w.L, w.p)
    assert _field_rel(mixed, ref) <= 1e-5


@pytest.mark.parametrize("case", [
    dict(n=20000, seed=31, L=3, p=8),
    dict(n=40000, seed=32, L=4, p=8, clustered_frac=0.4),
    dict(n=15000, seed=33, L=3, p=5),
    dict(n=30000, seed=34, L=5, p=3, clustered_frac=0.3),
])
def test_tensor_core_m2l_within_fp32_budget(orc, case):
    # PETFMM3D_OPT_M2L_TC (the default for p <= 8): M2L on tcgen05 with TF32
    # hi/lo operands; the same 1e-5 budget against the FP64 path, and close
    # to the SIMT GEMM M2L (option 0)
    from paper_0905_2637_gb300 import fmm3d
    w = W.tiny3d(case["n"], case["seed"], L=case["L"], p=case["p"], dtype="f32",
                 clustered_frac=case.get("clustered_frac", 0.0))
    ctx = _ctx(w, "mixed")
    ctx.set_option(fmm3d.PETFMM3D_OPT_M2L_TC, 1)
    rc, tc = _run(w, "mixed", ctx)
    ctx.close()
    assert rc == 0
    ctx = _ctx(w, "mixed")
    ctx.set_option(fmm3d.PETFMM3D_OPT_M2L_TC, 0)
    rc, simt = _run(w, "mixed", ctx)
    ctx.close()
    assert rc == 0
    rc, fp64 = _run(w, "fp64")
    assert rc == 0
    assert _rel(tc[0], fp64[0]) <= 1e-5
    assert _field_rel(tc, fp64) <= 1e-5
    assert _field_rel(tc, simt) <= 1e-5


def test_tensor_core_m2l_at_the_bench_size():
    # uniform3d-2M (2^21 charges, L = 5, p = 8): some 200 (source class,
    # offset) pairs reach each local expansion, the longest sums of the
    # tensor-core path; the potential is the more sensitive output
    w = W.uniform3d()
    rc, tc = _run(w, "mixed")
    assert rc == 0
    rc, fp64 = _run(w, "fp64")
    assert rc == 0
    assert _rel(tc[0], fp64[0]) <= 1e-5
    assert _field_rel(tc, fp64) <= 1e-5


def test_bitwise_reproducible_and_coincident_particles(orc):
    w = W.tiny3d(5000, 13, L=3, p=8, dtype="f32")
    w.x[1], w.y[1], w.z[1] = w.x[0], w.y[0], w.z[0]   # a coincident pair contributes 0
    ctx = _ctx(w, "mixed")
    a = _run(w, "mixed", ctx)[1]
    b = _run(w, "mixed", ctx)[1]
    ctx.close()
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    ref = orc.fmm3d(*w.as_f64(), w.domain, w.L, w.p)
    assert _field_rel(a, ref) <= 1e-5


def test_pair_across_a_leaf_face_closer_than_fp32():
    # Two FP64 particles 1e-13 apart on either side of the face x = 1/2
    # (leaves 3 and 4 at L = 3): their FP32 leaf coordinates are +-1/2, so
    # without the record cap the mixed near field would meet |d| = 0 between
    # two leaves and give inf.  The mixed path stays finite; every other
    # particle keeps its FP32 budget against the FP64 path.
    w = W.tiny3d(3000, 17, L=3, p=8, dtype="f64")
    w.x[0], w.y[0], w.z[0] = 0.5 - 1e-13, 0.3, 0.7
    w.x[1], w.y[1], w.z[1] = 0.5, 0.3, 0.7
    rc, mixed = _run(w, "mixed")
    assert rc == 0 and all(np.all(np.isfinite(a)) for a in mixed)
    rc, fp64 = _run(w, "fp64")
    assert rc == 0 and all(np.all(np.isfinite(a)) for a in fp64)
    rest = [a[2:] for a in mixed], [a[2:] for a in fp64]
    assert _field_rel(*rest) <= 1e-5


def test_empty_input_and_outside_particle_then_recovery():
    torch = G.torch_cuda()
    w = W.tiny3d(1000, 14, L=3, p=6, dtype="f32")
    ctx = _ctx(w, "mixed")
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.evaluate(e, e, e, e)
    assert ctx.sync() == 0
    bad = W.tiny3d(1000, 14, L=3, p=6, dtype="f32")
    bad.x[17] = 1.5
    from paper_0905_2637_gb300 import _lib
    with pytest.raises(_lib.PetfmmError) as err:
        _run(bad, "mixed", ctx)
    assert err.value.code == _lib.PETFMM_EDOMAIN
    rc, good = _run(w, "mixed", ctx)
    assert rc == 0 and all(np.all(np.isfinite(a)) for a in good)
    ctx.close()
