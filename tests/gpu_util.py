"""Helpers for the GPU tests: run the CUDA path through the C ABI on a
seeded workload and return numpy results."""
import numpy as np


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0905_2637_gb300 import _lib
    return _lib


def to_dev(arrs):
    torch = torch_cuda()
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def run(w, precision, L=None, p=None, sigma=None, domain=None, timing=False, ctx_out=None, poison=True,
        options=None):
    """One evaluation of workload w; returns (u, v) as float64 numpy arrays."""
    _lib = lib()
    L = w.L if L is None else L
    p = w.p if p is None else p
    ctx = _lib.Context(domain or w.domain, L, p, sigma or w.sigma, precision=precision, dtype=w.dtype)
    if timing:
        ctx.set_option(_lib.PETFMM_OPT_TIMING, 1)
    if poison:
        # any read of a coefficient this evaluation did not write turns into NaN
        ctx.set_option(_lib.PETFMM_OPT_POISON, 1)
    for opt, val in (options or {}).items():
        ctx.set_option(opt, val)
    x, y, g = to_dev((w.x, w.y, w.gamma))
    u, v = ctx.evaluate(x, y, g)
    rc = ctx.sync()
    assert rc == 0
    out = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    if ctx_out is not None:
        ctx_out.append(ctx)
    else:
        ctx.close()
    return out


def rel_l2(u, v, ur, vr):
    num = np.sum((u - ur) ** 2 + (v - vr) ** 2)
    den = np.sum(ur ** 2 + vr ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))
