"""Sharding one evaluation over several ranks: the tree cut of Sec. 4 with the
work and communication model of Sec. 5.1-5.2 (the partition and halo sets are
computed by the library's host code, ``petfmm_shard_*``), and the exchange of
halo data between ranks through ``torch.distributed``.

A rank owns the level-k subtrees ``partition`` assigns it.  Before it can
evaluate its particles it needs (``halo``): the particles of the other ranks'
leaves adjacent to its leaves, the multipole expansions of the other ranks'
boxes at levels k+1..L in the interaction lists of its boxes, and the
level-k expansions of every subtree (all-gathered).  ``exchange`` moves
per-destination arrays with one ``all_to_all_single`` on whatever backend the
process group has (NCCL with device tensors between GPUs, gloo with host
tensors): halos go through each GPU's own memory or the collective library,
never through peer loads of another GPU's memory.

This module moves and indexes data; it holds none of the method's
arithmetic.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


class ShardRank(ctypes.Structure):
    _fields_ = [("work", ctypes.c_double), ("comm", ctypes.c_double),
                ("particles", ctypes.c_int64), ("subtrees", ctypes.c_int32),
                ("first_subtree", ctypes.c_int32), ("last_subtree", ctypes.c_int32)]


_SIGS = False


def _lib_sigs():
    global _SIGS
    lib = _lib.load()
    if not _SIGS:
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        for name, res, args in (
                ("petfmm_shard_weights", I, [I, I, I, P, P]),
                ("petfmm_shard_comm", I, [I, I, D, P, P]),
                ("petfmm_shard_partition", I, [I, I, I, P, I, P, ctypes.POINTER(ShardRank)]),
                ("petfmm_shard_halo", I, [I, I, P, I, P, I64, P, I64, P, P])):
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _SIGS = True
    return lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def weights(L, k, order, leaf_counts):
    """Work (Eq. 13-15) of each of the 4^k subtrees."""
    lib = _lib_sigs()
    lc = _u32(leaf_counts)
    assert lc.size == 1 << (2 * L)
    out = np.zeros(1 << (2 * k), np.float64)
    _lib._ck(lib.petfmm_shard_weights(L, k, order, lc.ctypes.data, out.ctypes.data),
             "petfmm_shard_weights")
    return out


def comm(L, k, alpha=1.0):
    """(lateral, diagonal) expansion terms between neighbour subtrees."""
    lib = _lib_sigs()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib._ck(lib.petfmm_shard_comm(L, k, float(alpha), ctypes.byref(a), ctypes.byref(b)),
             "petfmm_shard_comm")
    return a.value, b.value


def partition(L, k, order, leaf_counts, nranks):
    """owner[s] (rank of level-k subtree s) and a per-rank summary."""
    lib = _lib_sigs()
    lc = _u32(leaf_counts)
    owner = np.zeros(1 << (2 * k), np.int32)
    ranks = (ShardRank * nranks)()
    _lib._ck(lib.petfmm_shard_partition(L, k, order, lc.ctypes.data, int(nranks),
                                        owner.ctypes.data, ranks), "petfmm_shard_partition")
    summ = [{f: getattr(r, f) for f, _ in ShardRank._fields_} for r in ranks]
    return owner, summ


def halo(L, k, owner, rank):
    """(leaves, boxes): the other ranks' leaves rank needs the particles of,
    and the (level, box) pairs it needs the multipole expansions of."""
    lib = _lib_sigs()
    own = np.ascontiguousarray(owner, dtype=np.int32)
    nl, nb = ctypes.c_int64(), ctypes.c_int64()
    _lib._ck(lib.petfmm_shard_halo(L, k, own.ctypes.data, int(rank), None, 0, None, 0,
                                   ctypes.byref(nl), ctypes.byref(nb)), "petfmm_shard_halo")
    leaves = np.zeros(max(nl.value, 1), np.int32)
    boxes = np.zeros((max(nb.value, 1), 2), np.int32)
    _lib._ck(lib.petfmm_shard_halo(L, k, own.ctypes.data, int(rank), leaves.ctypes.data, nl.value,
                                   boxes.ctypes.data, nb.value, ctypes.byref(nl),
                                   ctypes.byref(nb)), "petfmm_shard_halo")
    return leaves[:nl.value], boxes[:nb.value]


def leaf_owner(L, k, owner):
    """Rank owning each leaf (Morton order)."""
    m = np.arange(1 << (2 * L), dtype=np.int64)
    return np.asarray(owner)[m >> (2 * (L - k))]


def exchange(dist, send, width, dtype, device="cpu"):
    """All-to-all of variable-length rows: send[q] is a (n_q, width) array for
    rank q (q = 0..world-1, empty rows allowed); returns the list of arrays
    received from each rank.  Two collectives: the counts, then the rows."""
    import torch
    world = dist.get_world_size()
    counts = torch.tensor([int(np.asarray(send[q]).shape[0]) for q in range(world)],
                          dtype=torch.int64, device=device)
    recv_counts = torch.empty_like(counts)
    dist.all_to_all_single(recv_counts, counts)
    sc = counts.tolist()
    rc = recv_counts.tolist()
    flat = np.concatenate([np.asarray(send[q], dtype=dtype).reshape(-1, width) for q in range(world)]
                          + [np.zeros((0, width), dtype)])
    out = torch.empty((sum(rc), width), dtype=torch.from_numpy(np.zeros(0, dtype)).dtype,
                      device=device)
    dist.all_to_all_single(out, torch.from_numpy(np.ascontiguousarray(flat)).to(device), rc, sc)
    res, o = [], 0
    host = out.cpu().numpy()
    for q in range(world):
        res.append(host[o:o + rc[q]])
        o += rc[q]
    return res
