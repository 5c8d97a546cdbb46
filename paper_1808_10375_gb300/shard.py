"""View-sharded DM iteration through the C ABI.

Sec. III of the paper spreads the scan's views almost evenly over GPUs: each
rank runs the exit-wave update (Eq. 3) on its own views, and the sums over all
views in Eq. 5 and Eq. 4 are formed by reducing per-rank partial sums (the
paper's MPI reduce and broadcast).  Here a shard is a dm context that holds a
contiguous range of the views; ``sharded_iteration`` runs one iteration over
the shards a process holds, summing the partial sums over those shards and
then over processes with ``allreduce`` (for instance ``torch.distributed``
with gloo or NCCL; the identity when there is a single process).

Every step of the method runs in the library; this module only orders the
calls and adds the partial sums.  The protocol is the one declared beside
dm_object_partials in include/dm.h.
"""
from __future__ import annotations

import numpy as np

from . import dm


def split_views(views: int, shards: int):
    """Contiguous, almost even view ranges, one per shard (Sec. III)."""
    if shards < 1 or views < shards:
        raise ValueError("need 1 <= shards <= views")
    base, extra = divmod(views, shards)
    out, start = [], 0
    for s in range(shards):
        stop = start + base + (1 if s < extra else 0)
        out.append(range(start, stop))
        start = stop
    return out


def torch_allreduce(group=None):
    """An ``allreduce(array) -> array`` summing a NumPy array over the ranks of
    an initialised torch.distributed process group (its backend moves the
    data: gloo on host tensors, NCCL on device tensors)."""
    import torch
    import torch.distributed as tdist

    def reduce(a):
        a = np.ascontiguousarray(a)
        backend = tdist.get_backend(group)
        t = torch.from_numpy(a.copy())
        if backend == "nccl":
            t = t.cuda()
        tdist.all_reduce(t, op=tdist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()

    return reduce


def _sum(parts, dtype, allreduce):
    acc = np.zeros(parts[0].shape, dtype=dtype)
    for p in parts:
        acc += np.asarray(p, dtype=dtype)
    return allreduce(acc) if allreduce is not None else acc


def sharded_iteration(ctxs, allreduce=None):
    """One DM iteration over shard contexts (n_inner = 1, probe updated).

    ``ctxs`` are the shard contexts of this process (same frame size, modes,
    object size and parameters).  Partial sums are added over them in FP64,
    then over processes by ``allreduce``.  Afterwards every shard holds the
    same object and probe; each keeps the exit waves of its own views."""
    if not ctxs:
        raise ValueError("no shard contexts")
    for c in ctxs:
        dm.dm_run_step(c, dm.DM_STEP_FOURIER)
    parts = [dm.dm_object_partials(c) for c in ctxs]
    num = _sum([p[0] for p in parts], np.complex128, allreduce)
    den = _sum([p[1] for p in parts], np.float64, allreduce)
    for c in ctxs:
        dm.dm_object_apply(c, num, den)
    parts = [dm.dm_probe_partials(c) for c in ctxs]
    pnum = _sum([p[0] for p in parts], np.float64, allreduce)
    pden = _sum([p[1] for p in parts], np.float64, allreduce)
    for c in ctxs:
        dm.dm_probe_apply(c, pnum, pden)
    ef = _sum([np.asarray(dm.dm_fourier_error_partials(c)) for c in ctxs], np.float64, allreduce)
    for c in ctxs:
        dm.dm_finish_iteration(c, ef)
