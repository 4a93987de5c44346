"""petfmm_tree_noalloc: the tree build for callers that cannot allocate
device memory (their allocator owns the GPU, or they run under a fixed memory
budget).  Its keys, permutation and leaf starts must equal what the regular
entry point (petfmm_evaluate + petfmm_debug_tree) produces on the same input,
bit for bit (integer outputs), on two calls in a row -- the second call runs
on a static scratch array that still holds the first call's data.

This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import gpu_util as G
from paper_0905_2637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, w, stream):
    torch = G.torch_cuda()
    fn = lib.load().petfmm_tree_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lib.Domain), ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    x, y = G.to_dev((w.x, w.y))
    keys = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    perm = torch.zeros(w.n, dtype=torch.int32, device="cuda")
    start = torch.zeros((1 << (2 * w.L)) + 1, dtype=torch.int32, device="cuda")
    dom = lib.Domain(*map(float, w.domain))
    dt = lib.PETFMM_F32 if w.dtype == "f32" else lib.PETFMM_F64
    torch.cuda.synchronize()
    rc = fn(ctypes.byref(dom), w.L, dt, w.n, x.data_ptr(), y.data_ptr(), keys.data_ptr(),
            perm.data_ptr(), start.data_ptr(), ctypes.c_void_p(stream))
    return rc, keys.cpu().numpy().view(np.uint32), perm.cpu().numpy().view(np.uint32), \
        start.cpu().numpy().view(np.uint32)


def _regular(lib, w):
    ctx = lib.Context(w.domain, w.L, w.p, w.sigma, precision="mixed", dtype=w.dtype)
    x, y, g = G.to_dev((w.x, w.y, w.gamma))
    ctx.evaluate(x, y, g)
    assert ctx.sync() == 0
    out = ctx.debug_tree(w.n)
    ctx.close()
    return out


def test_noalloc_tree_matches_regular_entry_point_twice():
    lib = G.lib()
    torch = G.torch_cuda()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [W.tiny(300_000, 41, L=7, clustered_frac=0.5),
             W.tiny(1 << 20, 42, L=9, dtype="f32")]  # the maximum size
    for w in cases:  # two calls in a row, different sizes and data
        rc, keys, perm, start = _noalloc(lib, w, stream)
        assert rc == 0
        k2, p2, s2 = _regular(lib, w)
        assert np.array_equal(keys, k2)
        assert np.array_equal(perm, p2)
        assert np.array_equal(start, s2)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = G.lib()
    torch = G.torch_cuda()
    fn = lib.load().petfmm_tree_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lib.Domain), ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    dom = lib.Domain(0.0, 0.0, 1.0)
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    rc = fn(ctypes.byref(dom), 4, lib.PETFMM_F64, (1 << 20) + 1, p, p, None, p, p, None)
    assert rc == lib.PETFMM_ENOMEM
