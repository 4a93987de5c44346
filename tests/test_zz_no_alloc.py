"""petfmm_tree_noalloc: the tree build for callers that cannot allocate
device memory (their own caching allocator already holds the GPU, or they run
under a fixed, audited memory budget).

Its keys, permutation and leaf starts must equal the oracle's binning and
stable sort (Sec. 2.1, z-order of Sec. 5.1) bit for bit, and what the regular
entry point (petfmm_evaluate + petfmm_debug_tree) produces, on calls in a
row: the static scratch array keeps the previous call's data, so the cases
run small -> large -> small, FP64 and FP32 storage, both at the maximum size,
a call without keys, an empty call, and a call that reports a particle outside
the domain followed by a clean call.  Free device memory must not change
across calls.

This file is collected last on purpose: a run that stops at the first failure
has then already run every other test."""
import ctypes

import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fn(lib):
    fn = lib.load().petfmm_tree_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lib.Domain), ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


class _Bufs:
    """Caller-owned device inputs and outputs, allocated before the call."""

    def __init__(self, w, with_keys=True):
        torch = G.torch_cuda()
        self.x, self.y = G.to_dev((w.x, w.y))
        n = max(w.n, 1)
        # outputs start as garbage, so a word the call does not write shows up
        self.keys = torch.full((n,), -1, dtype=torch.int32, device="cuda") if with_keys else None
        self.perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        self.start = torch.full(((1 << (2 * w.L)) + 1,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()

    def result(self, n):
        k = self.keys[:n].cpu().numpy().view(np.uint32) if self.keys is not None else None
        return k, self.perm[:n].cpu().numpy().view(np.uint32), \
            self.start.cpu().numpy().view(np.uint32)


def _call(lib, w, b, stream):
    dom = lib.Domain(*map(float, w.domain))
    dt = lib.PETFMM_F32 if w.dtype == "f32" else lib.PETFMM_F64
    kp = b.keys.data_ptr() if b.keys is not None else None
    return _fn(lib)(ctypes.byref(dom), w.L, dt, w.n, b.x.data_ptr(), b.y.data_ptr(), kp,
                    b.perm.data_ptr(), b.start.data_ptr(), ctypes.c_void_p(stream))


def _oracle_tree(orc, w):
    xd, yd, _ = w.as_f64()
    _, _, key = orc.bin(xd, yd, w.domain, w.L)
    perm, start = orc.sort(key, w.L)
    return key, perm, start


def _regular(lib, w):
    ctx = lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype=w.dtype)
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    out = ctx.debug_tree(w.n)
    ctx.close()
    return out


def test_noalloc_tree_matches_oracle_and_regular_path_on_calls_in_a_row(orc):
    lib = G.lib()
    torch = G.torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    nmax = lib.PETFMM_NOALLOC_MAX_N if hasattr(lib, "PETFMM_NOALLOC_MAX_N") else 1 << 20
    cases = [W.tiny(300_000, 41, L=7, clustered_frac=0.5),
             W.tiny(nmax, 42, L=9, dtype="f32"),              # the maximum size, FP32
             W.tiny(nmax, 43, L=10, clustered_frac=0.3),      # the maximum size, FP64
             W.tiny(300_000, 44, L=7, dtype="f32")]           # small after large: stale tail
    for i, w in enumerate(cases):
        b = _Bufs(w)
        assert _call(lib, w, b, stream) == 0
        keys, perm, start = b.result(w.n)
        k0, p0, s0 = _oracle_tree(orc, w)
        assert np.array_equal(keys, k0)
        assert np.array_equal(perm, p0)
        assert np.array_equal(start, s0)
        if i < 2:  # the regular entry point agrees as well
            k2, p2, s2 = _regular(lib, w)
            assert np.array_equal(keys, k2) and np.array_equal(perm, p2)
            assert np.array_equal(start, s2)


def test_noalloc_without_keys_empty_and_after_a_domain_error(orc):
    lib = G.lib()
    torch = G.torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    # keys = NULL: perm and start still computed
    w = W.tiny(70_001, 45, L=6, clustered_frac=0.2)
    b = _Bufs(w, with_keys=False)
    assert _call(lib, w, b, stream) == 0
    _, perm, start = b.result(w.n)
    _, p0, s0 = _oracle_tree(orc, w)
    assert np.array_equal(perm, p0) and np.array_equal(start, s0)
    # n = 0: every leaf start is 0
    w0 = W.Workload("empty", np.zeros(0), np.zeros(0), np.zeros(0), 0.01, (0.0, 0.0, 1.0), 5, 8, "f64")
    b0 = _Bufs(w0)
    assert _call(lib, w0, b0, stream) == 0
    assert np.all(b0.result(0)[2] == 0)
    # a particle outside the closed domain: EDOMAIN, and the next call is clean
    wb = W.tiny(5_000, 46, L=4)
    xb = wb.x.copy()
    xb[1234] = 1.5
    bad = W.Workload("outside", xb, wb.y, wb.gamma, wb.sigma, wb.domain, wb.L, wb.p, wb.dtype)
    assert _call(lib, bad, _Bufs(bad), stream) == lib.PETFMM_EDOMAIN
    b = _Bufs(wb)
    assert _call(lib, wb, b, stream) == 0
    keys, perm, start = b.result(wb.n)
    k0, p0, s0 = _oracle_tree(orc, wb)
    assert np.array_equal(keys, k0) and np.array_equal(perm, p0) and np.array_equal(start, s0)


def test_noalloc_leaves_free_device_memory_unchanged():
    lib = G.lib()
    torch = G.torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    w = W.tiny(500_000, 47, L=8, dtype="f32", clustered_frac=0.4)
    b = _Bufs(w)
    assert _call(lib, w, b, stream) == 0      # first call: module load, address lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(lib, w, b, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = G.lib()
    torch = G.torch_cuda()
    fn = _fn(lib)
    dom = lib.Domain(0.0, 0.0, 1.0)
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    rc = fn(ctypes.byref(dom), 4, lib.PETFMM_F64, (1 << 20) + 1, p, p, None, p, p, None)
    assert rc == lib.PETFMM_ENOMEM
    assert fn(ctypes.byref(dom), 0, lib.PETFMM_F64, 10, p, p, None, p, p, None) == lib.PETFMM_EINVAL
