"""The FP64 oracle iteration with its views spread over host processes.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): used by ``tests/`` and
by the CPU-baseline leg of ``bench.py`` to run the oracle on every host core.

Sec. III of the paper spreads the views of a scan over ranks: each rank
applies Eq. 3 to its own views and the sums over views in Eq. 5 and Eq. 4
are formed by adding per-rank partial sums.  This module does the same with
worker processes (started with ``spawn``, each single-threaded) that keep the
exit waves of a contiguous range of views in their own memory.  Every step
of the method is a call into ``oracle.dm`` (``fourier_update_view``,
``field_products``, ``object_patch``); this module only splits the views,
adds the partial sums in the parent and applies the two divisions of Eq. 5
and Eq. 4 exactly as ``oracle.dm.object_update`` / ``probe_update`` do.

One ``iterate()`` equals ``oracle.dm.dm_iteration`` (Gauss-Seidel order, one
inner pass, probe updated) up to the order of the floating-point sums.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np


def _attach(spec):
    name, shape, dtype = spec
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _half(x):
    """Round complex values to complex half (IEEE binary16 parts, nearest even)."""
    return x.real.astype(np.float16).astype(np.float64) + 1j * x.imag.astype(np.float16).astype(np.float64)


def _worker(conn, a, b, specs, beta, keep, round_start):
    """Holds psi of views [a, b) (or, with keep=False, recomputes it from the
    initial P O when it is needed again); answers the parent's requests.
    With round_start the initial exit waves are rounded to complex half (the
    start of the mixed-precision form)."""
    from oracle import dm as odm
    handles = [_attach(s) for s in specs]
    inten, pos, probe, obj = (h[1] for h in handles)
    n = probe.shape[-1]
    psi = None
    start = None      # (probe, object) the single Fourier step started from (keep=False)

    def psi0_of(pr, ob, j):
        p0 = odm.field_products(pr, ob, pos[j])
        return _half(p0) if round_start else p0

    def psi_new_of(i, j):
        psi0 = psi0_of(start[0], start[1], j)
        return odm.fourier_update_view(psi0, start[0], start[1], pos[j], inten[j].astype(np.float64), beta)[0]

    try:
        while True:
            msg = conn.recv()
            op = msg[0]
            if op == "init":          # psi = P O on every footprint (Sec. II)
                if keep:
                    psi = np.stack([psi0_of(probe, obj, j) for j in range(a, b)])
                conn.send(None)
            elif op == "fourier":     # Eq. 3 on own views, Eq. 5 numerator band
                if not keep:
                    if start is not None:
                        raise RuntimeError("keep=False runs one iteration from P O")
                    start = (probe.copy(), obj.copy())
                r0 = int(pos[a:b, 0].min())
                r1 = int(pos[a:b, 0].max()) + n
                num = np.zeros((r1 - r0, obj.shape[1]), np.complex128)
                pc = np.conj(probe)
                ef = isum = d2 = n2 = 0.0
                for i, j in enumerate(range(a, b)):
                    old = psi[i] if keep else psi0_of(probe, obj, j)
                    new, e, s = odm.fourier_update_view(old, probe, obj, pos[j], inten[j].astype(np.float64), beta)
                    d2 += float(np.sum(np.abs(new - old) ** 2))
                    n2 += float(np.sum(np.abs(new) ** 2))
                    if keep:
                        psi[i] = new
                    ef += e
                    isum += s
                    r, c = int(pos[j, 0]), int(pos[j, 1])
                    num[r - r0:r - r0 + n, c:c + n] += np.sum(pc * new, axis=0)
                conn.send((r0, num, ef, isum, d2, n2))
            elif op == "probe":       # Eq. 4 partial sums with the current (new) object
                num = np.zeros(probe.shape, np.complex128)
                den = np.zeros((n, n))
                for i, j in enumerate(range(a, b)):
                    op_ = odm.object_patch(obj, pos[j], n)
                    num += np.conj(op_)[None] * (psi[i] if keep else psi_new_of(i, j))
                    den += np.abs(op_) ** 2
                conn.send((num, den))
            elif op == "sample":      # psi at probe pixels (uy, ux) of every own view
                uy, ux = msg[1], msg[2]
                conn.send(psi[:, :, uy, ux])
            else:
                conn.send(None)
                return
    finally:
        for shm, _ in handles:
            shm.close()


class ProcessDM:
    """Oracle DM over ``workers`` processes, from the exit waves psi = P O of
    the initial estimates; ``probe``/``obj`` hold the current estimates
    (FP64).  With ``keep_psi=False`` the workers store no exit waves and
    recompute the new ones for Eq. 4 (one iteration only, for scans whose
    FP64 exit waves do not fit in host memory).  With ``round_start`` the
    initial exit waves are rounded to complex half, as the mixed-precision
    form stores them.  Use as a context manager."""

    def __init__(self, intensities, pos, probe, obj, workers=None, beta=0.8, delta_rel=1e-6, keep_psi=True,
                 round_start=False):
        self.jn = int(np.asarray(pos).shape[0])
        self.n = probe.shape[-1]
        self.delta_rel = delta_rel
        self.workers = max(1, min(workers or os.cpu_count() or 1, self.jn))
        arrays = [np.ascontiguousarray(intensities), np.ascontiguousarray(np.asarray(pos).astype(np.int64)),
                  np.ascontiguousarray(probe, np.complex128), np.ascontiguousarray(obj, np.complex128)]
        self._shm, specs, views = [], [], []
        for arr in arrays:
            shm = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
            v = np.ndarray(arr.shape, arr.dtype, buffer=shm.buf)
            v[...] = arr
            self._shm.append(shm)
            specs.append((shm.name, arr.shape, arr.dtype))
            views.append(v)
        self._inten, self.pos, self.probe, self.obj = views
        bounds = np.linspace(0, self.jn, self.workers + 1).astype(int)
        ctx = mp.get_context("spawn")
        self._procs, self._conns = [], []
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            for a, b in zip(bounds[:-1], bounds[1:]):
                parent, child = ctx.Pipe()
                p = ctx.Process(target=_worker, args=(child, int(a), int(b), specs, beta, keep_psi, round_start), daemon=True)
                p.start()
                self._procs.append(p)
                self._conns.append(parent)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self._ask(("init",))

    def _ask(self, msg):
        for c in self._conns:
            c.send(msg)
        return [c.recv() for c in self._conns]

    def iterate(self):
        """One DM iteration (Eq. 3, Eq. 5, Eq. 4, Eq. 6); returns the metrics
        dict of oracle.dm.dm_iteration."""
        from oracle import dm as odm
        h, w = self.obj.shape
        obj0 = self.obj.copy()
        probe0 = self.probe.copy()
        num = np.zeros((h, w), np.complex128)
        ef = isum = d2 = n2 = 0.0
        for r0, band, e, s, a, b in self._ask(("fourier",)):
            num[r0:r0 + band.shape[0]] += band
            ef += e
            isum += s
            d2 += a
            n2 += b
        den = odm.object_denominator(self.probe, self.pos, (h, w))
        cov = den > 0
        new = obj0.copy()
        new[cov] = num[cov] / (den[cov] + self.delta_rel * den.max())
        self.obj[...] = new
        pnum = np.zeros(self.probe.shape, np.complex128)
        pden = np.zeros((self.n, self.n))
        for a, b in self._ask(("probe",)):
            pnum += a
            pden += b
        pnew = probe0.copy()
        pc = pden > 0
        pnew[:, pc] = pnum[:, pc] / (pden[pc] + self.delta_rel * pden.max())
        self.probe[...] = pnew
        return {"eps_obj": odm.rel_change(self.obj, obj0),
                "eps_probe": [odm.rel_change(self.probe[k], probe0[k]) for k in range(self.probe.shape[0])],
                "fourier_err": float(np.sqrt(ef / isum)) if isum > 0 else 0.0,
                "eps_psi": float(np.sqrt(d2 / n2)) if n2 > 0 else 0.0}

    def psi_at(self, uy, ux):
        """The exit waves of every view at probe pixels (uy, ux): [J, M, U]
        (keep_psi=True only)."""
        return np.concatenate(self._ask(("sample", np.asarray(uy), np.asarray(ux))))

    def close(self):
        if self._conns:
            try:
                self._ask(("stop",))
            except (EOFError, OSError, BrokenPipeError):
                pass
            for p in self._procs:
                p.join(timeout=10)
                if p.is_alive():
                    p.terminate()
            self._conns, self._procs = [], []
        # keep the estimates readable once the shared blocks are gone
        self.probe, self.obj, self.pos = self.probe.copy(), self.obj.copy(), self.pos.copy()
        self._inten = None
        for shm in self._shm:
            shm.close()
            shm.unlink()
        self._shm = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
