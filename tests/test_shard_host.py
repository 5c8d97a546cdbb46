"""Host-side logic of the view-sharded iteration, without a GPU: the view
split of Sec. III, the all-reduce wrapper over torch.distributed (gloo,
world size 2), and the decomposition it relies on, checked with the FP64
oracle: the per-shard numerators and denominators of Eq. 5 and Eq. 4, summed
over the shards by gloo, give the oracle's update of the whole scan."""
import os
import socket

import numpy as np
import pytest

from paper_1808_10375_gb300.shard import split_views


def test_split_views_is_contiguous_and_almost_even():
    for views in (1, 7, 100, 10000):
        for shards in (1, 2, 3, 8):
            if shards > views:
                with pytest.raises(ValueError):
                    split_views(views, shards)
                continue
            rs = split_views(views, shards)
            assert rs[0].start == 0 and rs[-1].stop == views
            assert all(a.stop == b.start for a, b in zip(rs, rs[1:]))
            sizes = [len(r) for r in rs]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_partials(psi, probe, obj, pos):
    """Numerators and denominators of Eq. 5 and Eq. 4 over the given views
    (the probe ones with `obj`), as the embedding and patch sums of Sec. III."""
    from oracle import dm as odm
    n = probe.shape[-1]
    onum = np.zeros(obj.shape, np.complex128)
    oden = np.zeros(obj.shape, np.float64)
    pnum = np.zeros(probe.shape, np.complex128)
    pden = np.zeros((n, n), np.float64)
    p2 = np.sum(np.abs(probe) ** 2, axis=0)
    for j in range(len(pos)):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        onum[r:r + n, c:c + n] += np.sum(np.conj(probe) * psi[j], axis=0)
        oden[r:r + n, c:c + n] += p2
        op = odm.object_patch(obj, pos[j], n)
        pnum += np.conj(op)[None] * psi[j]
        pden += np.abs(op) ** 2
    return onum, oden, pnum, pden


def _worker(rank, world, port, q):
    import torch.distributed as tdist
    from oracle import dm as odm
    from paper_1808_10375_gb300.shard import torch_allreduce
    from parity_util import case
    try:
        tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        reduce = torch_allreduce()
        s, p0, o0, psi0 = case(16, 2, (4, 4), 4, (30, 30), 31)
        psi = psi0.astype(np.complex128)
        probe = p0.astype(np.complex128)
        obj = o0.astype(np.complex128)
        mine = split_views(s.views, world)[rank]
        idx = np.arange(mine.start, mine.stop)
        onum, oden, _, _ = _shard_partials(psi[idx], probe, obj, s.pos[idx])
        onum, oden = reduce(onum), reduce(oden)
        o_new = obj.copy()
        cov = oden > 0
        o_new[cov] = onum[cov] / (oden[cov] + 1e-6 * oden.max())
        _, _, pnum, pden = _shard_partials(psi[idx], probe, o_new, s.pos[idx])
        pnum, pden = reduce(pnum), reduce(pden)
        p_new = probe.copy()
        cov = pden > 0
        p_new[:, cov] = pnum[:, cov] / (pden[cov] + 1e-6 * pden.max())
        o_ref = odm.object_update(psi, probe, obj, s.pos, 1e-6)
        p_ref = odm.probe_update(psi, probe, o_ref, s.pos, 1e-6)
        eo = np.linalg.norm(o_new - o_ref) / np.linalg.norm(o_ref)
        ep = np.linalg.norm(p_new - p_ref) / np.linalg.norm(p_ref)
        q.put((rank, float(eo), float(ep)))
        tdist.destroy_process_group()
    except Exception as e:  # pragma: no cover - reported by the parent
        q.put((rank, repr(e), None))


def test_gloo_shard_sums_reproduce_the_whole_scan_update():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for rank, eo, ep in res:
        assert isinstance(eo, float), eo
        assert eo <= 1e-12 and ep <= 1e-12, (rank, eo, ep)
