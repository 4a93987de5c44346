"""One evaluation sharded over 2 and 4 ranks by the tree cut of Sec. 4 (gloo
processes on the CPU): each rank owns the subtrees the z-order partition
gives it, receives only its halo -- the particles of foreign leaves next to
its leaves, the multipole expansions of foreign boxes in its interaction
lists, and every subtree's level-k expansion -- and evaluates its own
particles.  The union of the ranks' velocities must equal the single-process
FMM (the oracle's, FP64) to rounding: a leaf or box missing from a halo set
would change the result.

The per-rank arithmetic here uses the oracle's single operators (test
infrastructure); what is under test is the partition, the halo sets and the
exchange of the package's shard module."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

L, K, P_ORD = 5, 2, 10


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _centre(dom, l, m):
    x0, y0, W = dom
    r = W / (1 << l)
    ix = iy = 0
    for b in range(16):
        ix |= ((m >> (2 * b)) & 1) << b
        iy |= ((m >> (2 * b + 1)) & 1) << b
    return complex(x0 + (ix + 0.5) * r, y0 + (iy + 0.5) * r), ix, iy


def _workload():
    from paper_0905_2637_gb300 import workloads as W
    return W.tiny(3000, 21, L=L, p=P_ORD, clustered_frac=0.4)


def _rank_main(rank, ws, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        from paper_0905_2637_gb300 import shard
        w = _workload()
        dom, sig, p = w.domain, w.sigma, w.p
        _, _, key = oracle.bin(w.x, w.y, dom, L)
        counts = np.bincount(key, minlength=1 << (2 * L)).astype(np.uint32)
        owner, summ = shard.partition(L, K, p, counts, ws)
        lown = shard.leaf_owner(L, K, owner)
        mine = np.flatnonzero(lown[key] == rank)          # global indices of my particles
        halos = [shard.halo(L, K, owner, q) for q in range(ws)]
        # 1. particles of my leaves that other ranks' halos list
        rows = np.stack([w.x, w.y, w.gamma, np.arange(w.n, dtype=np.float64)], 1)
        send = []
        for q in range(ws):
            want = np.zeros(1 << (2 * L), bool)
            want[halos[q][0]] = True
            sel = mine[want[key[mine]]] if q != rank else np.zeros(0, np.int64)
            send.append(rows[sel])
        got = shard.exchange(dist, send, 4, np.float64)
        halo_rows = np.concatenate(got)
        # 2. my multipole expansions, levels K..L (leaves by P2M, then M2M)
        me = {}
        for m in np.unique(key[mine]):
            sel = mine[key[mine] == m]
            zc, _, _ = _centre(dom, L, int(m))
            me[(L, int(m))] = oracle.p2m(w.x[sel], w.y[sel], w.gamma[sel], zc, p)
        for l in range(L - 1, K - 1, -1):
            for (ll, m), a in [(kk, v) for kk, v in me.items() if kk[0] == l + 1]:
                par = m >> 2
                zp, _, _ = _centre(dom, l, par)
                zc, _, _ = _centre(dom, l + 1, m)
                me[(l, par)] = me.get((l, par), 0) + oracle.m2m(a, zc, zp)

        def me_rows(keys):
            out = [np.concatenate([[l, m], me[(l, m)].real, me[(l, m)].imag])
                   for (l, m) in keys if (l, m) in me]
            return np.array(out).reshape(-1, 2 + 2 * p)
        # 3. the expansions of my boxes in other ranks' interaction-list halos,
        #    and my level-K expansions to everyone
        send = []
        for q in range(ws):
            keys = [] if q == rank else [(int(l), int(m)) for l, m in halos[q][1]]
            keys += [(K, int(s)) for s in np.flatnonzero(owner == rank)] if q != rank else []
            send.append(me_rows(keys))
        for arr in shard.exchange(dist, send, 2 + 2 * p, np.float64):
            for r in arr:
                me[(int(r[0]), int(r[1]))] = r[2:2 + p] + 1j * r[2 + p:]
        # 4. the root tree (every rank for itself), then my subtrees' local
        #    expansions: M2L over the interaction list + L2L from the parent
        for l in range(K - 1, -1, -1):
            for m in range(1 << (2 * (l + 1))):
                if (l + 1, m) in me:
                    zp, _, _ = _centre(dom, l, m >> 2)
                    zc, _, _ = _centre(dom, l + 1, m)
                    me[(l, m >> 2)] = me.get((l, m >> 2), 0) + oracle.m2m(me[(l + 1, m)], zc, zp)
        le = {}
        for l in range(2, L + 1):
            for m in range(1 << (2 * l)):
                if l > K and owner[m >> (2 * (l - K))] != rank:
                    continue
                zt, ix, iy = _centre(dom, l, m)
                b = np.zeros(p, complex)
                for sx, sy in oracle.interaction_list(l, ix, iy):
                    sm = 0
                    for bit in range(16):
                        sm |= ((int(sx) >> bit) & 1) << (2 * bit) | ((int(sy) >> bit) & 1) << (2 * bit + 1)
                    if (l, sm) in me:  # empty boxes have no expansion (zero)
                        zs, _, _ = _centre(dom, l, sm)
                        b = b + oracle.m2l(me[(l, sm)], zs, zt)
                    elif l > K:
                        assert owner[sm >> (2 * (l - K))] == rank or \
                            counts[sm << (2 * (L - l)):(sm + 1) << (2 * (L - l))].sum() == 0, \
                            f"missing halo box {(l, sm)}"
                if l > 2 and (l - 1, m >> 2) in le:
                    zp, _, _ = _centre(dom, l - 1, m >> 2)
                    b = b + oracle.l2l(le[(l - 1, m >> 2)], zp, zt)
                le[(l, m)] = b
        # 5. my particles: far field (L2P) + near field over the 9 leaves,
        #    my own particles and the halo's
        px = np.concatenate([w.x[mine], halo_rows[:, 0]])
        py = np.concatenate([w.y[mine], halo_rows[:, 1]])
        pg = np.concatenate([w.gamma[mine], halo_rows[:, 2]])
        pidx = np.concatenate([mine, halo_rows[:, 3].astype(np.int64)])
        pkey = key[pidx]
        res = []
        for m in np.unique(key[mine]):
            zl, ix, iy = _centre(dom, L, int(m))
            near = []
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    x2, y2 = ix + dx, iy + dy
                    if 0 <= x2 < (1 << L) and 0 <= y2 < (1 << L):
                        mm = 0
                        for bit in range(16):
                            mm |= ((x2 >> bit) & 1) << (2 * bit) | ((y2 >> bit) & 1) << (2 * bit + 1)
                        near.append(np.flatnonzero(pkey == mm))
            near = np.concatenate(near)
            tgt = np.flatnonzero(pkey[near] == m)
            tgt = tgt[np.isin(pidx[near][tgt], mine)]
            un, vn = oracle.direct(px[near], py[near], pg[near], sig, targets=tgt)
            for t, a_u, a_v in zip(tgt, un, vn):
                wv = oracle.l2p(le[(L, int(m))], zl, complex(px[near][t], py[near][t]))
                res.append((pidx[near][t], a_u + wv.imag / (2 * np.pi), a_v + wv.real / (2 * np.pi)))
        queue.put((rank, res, summ[rank]["particles"], len(mine)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])
def test_sharded_evaluation_equals_single_process_fmm(orc, ws):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=300) for _ in range(ws)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    w = _workload()
    u, v = np.full(w.n, np.nan), np.full(w.n, np.nan)
    for rank, res, npart, nmine in out:
        assert npart == nmine  # the partition's count is the rank's particles
        for i, a_u, a_v in res:
            assert np.isnan(u[i])  # each particle evaluated by exactly one rank
            u[i], v[i] = a_u, a_v
    assert not np.any(np.isnan(u))
    ur, vr = orc.fmm(w.x, w.y, w.gamma, w.domain, L, w.p, w.sigma)
    rel = np.sqrt(np.sum((u - ur) ** 2 + (v - vr) ** 2) / np.sum(ur ** 2 + vr ** 2))
    assert rel <= 1e-12
