"""Benchmark of the multi-mode difference-map iteration on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one DM iteration (Eq. 3, Eq. 5, Eq. 4, Eq. 6) over every view and
probe mode of the 8-mode 256x256-frame workload (10,000 views, 2100x2100
object; synthetic, seeded).  The metric is view*modes processed per second.

* value: device time (CUDA events on the library's stream) of K iterations
  with every input resident in HBM; the exit waves (42 GB) exceed L2, so no
  flush is needed between iterations.
* e2e: the same metric through the C ABI with host (pinned) buffers: dm_init
  from host memory, K iterations, object/probe/metrics back to the host, all
  inside the timed region; the bytes are reported per step.
* roofline: the persistent Fourier-step kernel, the dominant one, timed with
  CUDA events around each of its launches inside the timed region.
* cpu_baseline: the FP64 oracle on a bounded sample of the same workload on
  the host cores.
* --impl reference: the FP64 oracle itself, timed on the host cores, one
  bounded sample of views per step (there is no other implementation of the
  paper's method to run).

With N > 1 (torchrun) every rank runs an independent replica of the workload
(the method is run on one GPU per scan, no data is exchanged); the time is
the maximum over ranks and the value counts the views of all ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "view·modes/s per DM iteration"
UNIT = "view·modes/s"
WORKLOAD = "mm256"
WORKLOAD_DESC = ("8-mode difference map, 256x256 frames, 100x100 scan (10,000 views) at 18 px, "
                 "2100x2100 object, Hermite-Gauss probe modes, 1e7 photons/frame, FP32")
KERNELS_PER_ITER = 7   # fourier, obj gather, obj final, probe partial, probe sum, probe div, metrics


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--views", type=int, default=None, help="use only the first V views (small case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", type=int, default=0, metavar="V",
                    help="pick the Fourier-step plan with dm_autotune on the first V views before timing (0: the "
                         "default plan)")
    ap.add_argument("--form", choices=["auto", "strip", "split", "cluster"], default="auto",
                    help="Fourier-step form (auto: the context's choice, the split form for 256x256 frames with 8 "
                         "modes; after --autotune the autotuner's)")
    ap.add_argument("--psi", choices=["fp32", "fp16"], default="fp32",
                    help="exit-wave storage of the timed iteration (fp16: the mixed-precision form, no switch)")
    ap.add_argument("--cpu-views", type=int, default=600, help="views in the one-process oracle sample")
    ap.add_argument("--cpu-views-per-core", type=int, default=48,
                    help="views per worker process in the all-cores oracle sample")
    ap.add_argument("--ref-views-per-core", type=int, default=16,
                    help="--impl reference: views per worker process in each step's sample")
    ap.add_argument("--tte-iters", type=int, default=3000, help="tte: iteration limit of each DM run")
    ap.add_argument("--batch-iters", type=int, default=200, help="batch16: iterations of the convergence comparison")
    ap.add_argument("--judge-iters", type=int, default=50,
                    help="warmstart/tte: trial DM iterations from each start before the judge compares their "
                         "Fourier errors (after 10 the learned start led, but stalled later)")
    ap.add_argument("--tte-psi-switch", type=float, default=5e-5,
                    help="tte: Eq. 6 object change below which the mixed form returns to complex64 exit waves")
    ap.add_argument("--tte-train-steps", type=int, default=3000, help="tte: training steps of the warm-start "
                    "network (0: no warm-started run)")
    ap.add_argument("--workload", choices=["mm256", "mm128", "batch16", "dft256", "warmstart", "embed", "tte"],
                    default="mm256",
                    help="mm256: the 8-mode 256x256 scan (the headline); mm128: the 4-mode 128x128 scan "
                         "(2,500 views); batch16: sixteen uneven scans "
                         "advanced as one batch; dft256: the batched 2-D DFT in both precision forms; "
                         "warmstart: train the warm-start network, judge its start with DM; embed: the "
                         "object embedding fused into the exit-wave update against a separate pass; tte: "
                         "time to object error 1e-3 of plain FP32 DM from a flat, a random and a learned start")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        # Wait (at most 10 s) for the first sample, so that nvidia-smi's own
        # start-up is over before the timed region begins; that sample is
        # taken before the region and is left out of the summary.
        if self.proc is not None:
            import select
            ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
            if ready:
                self.proc.stdout.readline()
        time.sleep(0.05)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local]
    return local


WORKLOADS = {
    "mm256": WORKLOAD_DESC,
    "mm128": ("4-mode difference map, 128x128 frames, 50x50 scan (2,500 views) at 10 px, 640x640 object, "
              "Hermite-Gauss probe modes 0.6/0.25/0.1/0.05, 1e7 photons/frame, FP32"),
}


def make_inputs(views, device, name=WORKLOAD):
    import torch
    from synth import make_scan, initial_guess
    s = make_scan(name, backend="torch", device=device, views=views)
    rng = np.random.default_rng(s.meta["seed"] + 1)
    p0, o0 = initial_guess(s, rng, kind="perturbed")
    return s, p0.astype(np.complex64), o0.astype(np.complex64)


FORM_KERNEL = {"strip": "dm_fourier.cu", "split": "dm_fourier_split.cu", "cluster": "dm_fourier_cluster.cu"}
FORM_TRAFFIC = {"strip": "fourier_mm256_traffic.json", "split": "fourier_split_mm256_traffic.json"}
FORM_KERNEL_NAME = {
    "strip": "k_fourier (persistent Fourier step, Eq. 3, strip form)",
    "split": "k_fourier_split (persistent Fourier step, Eq. 3, split-column form)",
    "cluster": "k_fourier_cluster (Fourier step, Eq. 3, one cluster per view, frames in shared memory)",
}


def kernel_source_hash(form="strip"):
    """Hash of the sources of one form of the Fourier-step kernel; a stored
    DRAM-traffic figure is used only while it matches."""
    import hashlib
    h = hashlib.sha256()
    for f in (FORM_KERNEL[form], "dm_fft.cuh", "dm_kernels.h", "dm_psi.cuh", "dm_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_1808_10375_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(views, form="strip"):
    """DRAM bytes of one Fourier-step launch of the given form from the
    committed ncu summary, scaled from its capture size to `views` views, or
    None if the kernel changed since the capture."""
    if form not in FORM_TRAFFIC:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", FORM_TRAFFIC[form])) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash(form):
        return None
    return d["dram_bytes_per_launch"] * views / d["views"]


def fourier_bytes_per_view(n, m, psi_bytes=8):
    """Algorithmic bytes of the Fourier step (exit wave, FFTs, modulus
    projection, psi update) per view: psi read and write (psi_bytes per
    complex value per mode each: 8 for complex64, 4 for the complex-half
    storage of the mixed-precision form) and I read (4 B per pixel)."""
    return (2 * psi_bytes * m + 4) * n * n


def object_source_bytes_per_view(n):
    """Bytes per view of the object source c_j that the Fourier kernel also
    writes (8 B per pixel): an intermediate of this implementation, which the
    object gather reads instead of psi."""
    return 8 * n * n


def fourier_flops_per_view(n, m):
    """FFT operations of the Fourier step per view, by the usual count of
    5 L log2(L) real operations per complex transform of L points: two 2-D
    transforms (forward and inverse) of L = N^2 points per mode."""
    return 2 * 5 * n * n * int(round(math.log2(n * n))) * m


def iteration_bytes_per_view(n, m, psi_bytes=8):
    """Algorithmic bytes of one DM iteration per view: psi read and written by
    the Fourier step, read by the object and by the probe update, I read."""
    return (4 * psi_bytes * m + 4) * n * n


def rank_collectives(pg, device):
    """(barrier, max_over_ranks) for the replicas: every rank times its own
    replica and the job's time is the slowest rank's.  ``pg`` is
    torch.distributed (any backend) or None for one process."""
    def barrier():
        if pg is not None:
            pg.barrier()

    def max_over_ranks(x):
        if pg is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def job_throughput(world, views, modes, steps, seconds):
    """view*modes per second of the whole job: every rank advances its own
    replica of ``views`` views by ``steps`` iterations in ``seconds`` (the
    maximum over ranks)."""
    return world * views * modes * steps / seconds


def oracle_sample(s, p0, o0, views):
    """One oracle iteration over the first `views` views (same frames, modes
    and object); returns seconds."""
    from oracle import dm as odm
    import torch
    pos = s.pos[:views]
    inten = s.intensities[:views]
    inten = inten.cpu().numpy() if isinstance(inten, torch.Tensor) else np.asarray(inten)
    inten = inten.astype(np.float64)
    p = p0.astype(np.complex128)
    o = o0.astype(np.complex128)
    psi = odm.init_exit_waves(p, o, pos)
    t0 = time.perf_counter()
    odm.dm_iteration(psi, p, o, pos, inten)
    return time.perf_counter() - t0


def host_cpu():
    """(nproc, CPU model) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return os.cpu_count() or 1, model


def oracle_sample_cores(s, p0, o0, views, workers, iters=1):
    """Oracle iterations over the first `views` views with the views split
    over `workers` processes (oracle.parallel, as Sec. III splits them over
    ranks); returns seconds per iteration (the exit waves P O are built
    before the clock starts)."""
    from oracle.parallel import ProcessDM
    import torch
    inten = s.intensities[:views]
    inten = inten.cpu().numpy() if isinstance(inten, torch.Tensor) else np.asarray(inten)
    with ProcessDM(np.ascontiguousarray(inten, np.float32), s.pos[:views], p0.astype(np.complex128),
                   o0.astype(np.complex128), workers=workers) as pdm:
        t0 = time.perf_counter()
        for _ in range(iters):
            pdm.iterate()
        return (time.perf_counter() - t0) / iters


def cpu_baseline_line(s, p0, o0, j, m, args):
    """The oracle on the host cores: one process over a view sample and all
    cores (processes over views) over a larger one, both scaled to
    view-modes per second."""
    nproc, model = host_cpu()
    cv = min(args.cpu_views, j)
    secs1 = oracle_sample(s, p0, o0, cv)
    workers = max(1, nproc)
    cvn = min(j, args.cpu_views_per_core * workers)
    secsn = oracle_sample_cores(s, p0, o0, cvn, workers)
    return {"value": cvn * m / secsn, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"one FP64 oracle iteration over the first {cvn} views of the same scan with the views "
                      f"split over {workers} worker processes (oracle.parallel: Eq. 3 and the Eq. 4/5 partial "
                      f"sums in the workers, the divisions in the parent): {secsn:.1f} s",
            "one_core": {"value": cv * m / secs1, "cores": 1,
                         "sample": f"one FP64 oracle iteration (NumPy, one process) over the first {cv} views: "
                                   f"{secs1:.1f} s"},
            "nproc": nproc, "cpu_model": model}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    nproc, model = host_cpu()
    workers = max(1, nproc)
    views = max(workers, args.ref_views_per_core * workers)
    s, p0, o0 = make_inputs(views, dev)
    m = s.modes
    from oracle.parallel import ProcessDM
    inten = s.intensities
    inten = inten.cpu().numpy() if isinstance(inten, torch.Tensor) else np.asarray(inten)
    with ProcessDM(np.ascontiguousarray(inten, np.float32), s.pos, p0.astype(np.complex128),
                   o0.astype(np.complex128), workers=workers) as pdm:
        for _ in range(args.warmup):
            pdm.iterate()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pdm.iterate()
        tot = time.perf_counter() - t0
    value = views * m * args.steps / tot
    sample = (f"one FP64 oracle iteration per step over the first {views} views of {WORKLOAD}, the views split "
              f"over {workers} worker processes (oracle.parallel); nproc {nproc}, {model}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "views_per_step": views, "modes": m, "n": s.n,
                   "object": list(s.obj_shape)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                         "nproc": nproc, "cpu_model": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch16(args, rank, local):
    """Sixteen uneven scans: each run alone (dm_iterate, one after another)
    and as one batch (one persistent Fourier launch per frame size,
    CUDA-graph replay), after each context's autotuner has picked its Fourier
    plan.  The value is the batch's view*modes per second over all scans.
    Also: the per-scan convergence over --batch-iters iterations, batched
    against alone (Eq. 6 and the Fourier error of every iteration, final
    object and probe)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm
    from synth import batch16_configs, initial_guess
    torch.cuda.set_device(local)
    ctxs, vm = [], []
    for cfg in batch16_configs():
        sc = make_scan_cfg(cfg)
        rng = np.random.default_rng(cfg["seed"] + 1)
        p0, o0 = initial_guess(sc, rng, kind="perturbed")
        h, w = sc.obj_shape
        params = dm.dm_params_default(n=sc.n, modes=sc.modes, views=sc.views, obj_h=h, obj_w=w, beta=0.8)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        c = dm.dm_init(params, dev(sc.pos), sc.intensities, dev(p0.astype(np.complex64)),
                       dev(o0.astype(np.complex64)))
        dm.dm_autotune(c, sample_views=min(sc.views, 400))
        ctxs.append(c)
        vm.append(sc.views * sc.modes)
    total_vm = float(sum(vm))

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        for c in ctxs:
            dm.dm_sync(c)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    for c in ctxs:
        dm.dm_set_graph(c, True)
        dm.dm_iterate(c, args.warmup)
    t_alone = timed(lambda: [dm.dm_iterate(c, args.steps) for c in ctxs])
    b = dm.dm_batch_create(ctxs)
    dm.dm_batch_set_graph(b, True)
    dm.dm_batch_iterate(b, args.warmup)
    with ClockSampler(gpu_index(local)) as clk:
        t_batch = timed(lambda: dm.dm_batch_iterate(b, args.steps))
    dm.dm_batch_free(b)

    # sixteen small scans (64x64 frames, 100 views, 1-3 modes), where one scan
    # alone cannot fill the GPU
    small, svm = [], 0.0
    for i in range(16):
        cfg = dict(n=64, modes=1 + i % 3, grid=(10, 10), step=8, jitter=1, obj=(160, 160),
                   probe="gauss" if i % 3 == 0 else "hg", fwhm=32.0, photons=1e6, seed=3001 + i)
        sc = make_scan_cfg(cfg)
        p0s, o0s = initial_guess(sc, np.random.default_rng(cfg["seed"] + 1), kind="perturbed")
        prm = dm.dm_params_default(n=64, modes=sc.modes, views=sc.views, obj_h=160, obj_w=160, beta=0.8)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        c = dm.dm_init(prm, dev(sc.pos), sc.intensities, dev(p0s.astype(np.complex64)), dev(o0s.astype(np.complex64)))
        dm.dm_set_graph(c, True)
        dm.dm_iterate(c, args.warmup)
        small.append(c)
        svm += sc.views * sc.modes
    ts_alone = timed(lambda: [dm.dm_iterate(c, args.steps) for c in small])
    bs = dm.dm_batch_create(small)
    dm.dm_batch_set_graph(bs, True)
    dm.dm_batch_iterate(bs, args.warmup)
    ts_batch = timed(lambda: dm.dm_batch_iterate(bs, args.steps))
    dm.dm_batch_free(bs)
    for c in small:
        dm.dm_free(c)
    ferr = [dm.dm_get_error(c)[2] for c in ctxs]
    plans = [dm.dm_get_plan(c) for c in ctxs]
    for c in ctxs:
        dm.dm_free(c)

    # per-scan convergence over args.batch_iters iterations: every scan run
    # alone and the sixteen advanced together by the batch, from the same start
    def fresh():
        out = []
        for cfg in batch16_configs():
            sc = make_scan_cfg(cfg)
            rng = np.random.default_rng(cfg["seed"] + 1)
            p0, o0 = initial_guess(sc, rng, kind="perturbed")
            h, w = sc.obj_shape
            params = dm.dm_params_default(n=sc.n, modes=sc.modes, views=sc.views, obj_h=h, obj_w=w, beta=0.8)
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            out.append(dm.dm_init(params, dev(sc.pos), sc.intensities, dev(p0.astype(np.complex64)),
                                  dev(o0.astype(np.complex64))))
        return out
    hist = lambda c, n: [dm.dm_get_error(c, i) for i in range(n)]
    nb = args.batch_iters
    alone = fresh()
    for c in alone:
        # the batch runs each scan's Fourier step in the strip form, or in the
        # cluster form where that is the scan's own; the same form alone gives
        # the same arithmetic, so the monitors must agree exactly
        if dm.dm_get_fourier_form(c) == dm.DM_FOURIER_SPLIT:
            dm.dm_set_fourier_form(c, dm.DM_FOURIER_STRIP)
        dm.dm_iterate(c, nb)
    h_alone = [hist(c, nb) for c in alone]
    fin_alone = [(dm.dm_get_object(c), dm.dm_get_probe(c)) for c in alone]
    for c in alone:
        dm.dm_free(c)
    together = fresh()
    bt = dm.dm_batch_create(together)
    dm.dm_batch_iterate(bt, nb)
    dm.dm_batch_free(bt)
    h_tog = [hist(c, nb) for c in together]
    fin_tog = [(dm.dm_get_object(c), dm.dm_get_probe(c)) for c in together]
    for c in together:
        dm.dm_free(c)
    convergence = []
    for i in range(len(h_alone)):
        d_eo = max(abs(a[0] - b_[0]) / max(abs(a[0]), 1e-300) for a, b_ in zip(h_alone[i], h_tog[i]))
        d_ef = max(abs(a[2] - b_[2]) / max(abs(a[2]), 1e-300) for a, b_ in zip(h_alone[i], h_tog[i]))
        convergence.append({
            "scan": i, "eps_obj_first": h_alone[i][0][0], "eps_obj_last": h_alone[i][-1][0],
            "fourier_err_first": h_alone[i][0][2], "fourier_err_last": h_alone[i][-1][2],
            "max_rel_diff_eps_obj": d_eo, "max_rel_diff_fourier_err": d_ef,
            "object_identical": bool(np.array_equal(fin_alone[i][0], fin_tog[i][0])),
            "probe_identical": bool(np.array_equal(fin_alone[i][1], fin_tog[i][1]))})
    if rank == 0:
        line = {
            "metric": METRIC + ", sixteen scans batched", "value": total_vm * args.steps / t_batch, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch16: 16 seeded scans, frames 64/128/256, 400-6400 views, 1-8 modes, "
                                   "objects 454-1442 px", "scans": [list(x) for x in
                                                                    __import__("synth").BATCH16],
                       "view_modes_per_step": total_vm},
            "alone": {"value": total_vm * args.steps / t_alone, "ms_per_step": 1e3 * t_alone / args.steps,
                      "how": "dm_iterate on each scan in turn (CUDA-graph replay), same autotuned plans"},
            "batched_over_alone": t_alone / t_batch,
            "small16": {"scans": "16 scans of 64x64 frames, 100 views, 1-3 modes",
                        "batched": svm * args.steps / ts_batch, "alone": svm * args.steps / ts_alone,
                        "batched_over_alone": ts_alone / ts_batch, "unit": UNIT},
            "fourier_err_last": ferr,
            "plans": plans,
            "convergence": {"iterations": nb, "how": "each scan alone (dm_iterate, in the Fourier-step form the "
                                                    "batch runs for it: the strip form, or the cluster form where "
                                                    "that is the scan's own) and all sixteen in one batch "
                                                    "(dm_batch_iterate), from the same inputs; monitors of every "
                                                    "iteration compared", "scans": convergence},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_dft256(args, rank, local):
    """The batched 256 x 256 2-D DFT (dm_dft2) on the exit waves of the first
    1,000 views of the 8-mode workload (8,000 frames), in the FP32 register-FFT
    form and the two split-BF16 tensor-core forms (radix-16 stages on mma.sync;
    dense row GEMMs on tcgen05 with tensor-memory accumulators): frames per
    second, the tensor forms' tensor-core FLOP/s against the measured bf16
    peak, and each form's relative L2 error against numpy's FP64 FFT on a
    sample of the frames.  The line's value and roofline are the tcgen05
    form's."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm
    from synth import make_scan
    torch.cuda.set_device(local)
    views = args.views or 1000
    s = make_scan(WORKLOAD, backend="torch", device="cuda", views=views)
    p = torch.from_numpy(s.probe.astype(np.complex64)).cuda()
    o = torch.from_numpy(s.obj.astype(np.complex64)).cuda()
    pos = torch.from_numpy(s.pos.astype(np.int64)).cuda()
    ar = torch.arange(s.n, device="cuda")
    frames = torch.empty((views * s.modes, s.n, s.n), dtype=torch.complex64, device="cuda")
    for j0 in range(0, views, 100):
        j1 = min(views, j0 + 100)
        rr = pos[j0:j1, 0][:, None, None] + ar[None, :, None]
        cc = pos[j0:j1, 1][:, None, None] + ar[None, None, :]
        frames[j0 * s.modes:j1 * s.modes] = (p[None] * o[rr, cc][:, None]).reshape(-1, s.n, s.n)
    nf = frames.shape[0]
    work = torch.empty_like(frames)
    out = torch.empty_like(frames)
    sample = torch.arange(0, nf, max(1, nf // 48))[:48]
    ref = np.fft.fft2(frames[sample].cpu().numpy().astype(np.complex128))
    res = {}
    for prec, name in ((dm.DM_DFT_FP32, "fp32_fft"), (dm.DM_DFT_BF16X3, "bf16x3_tensor"),
                       (dm.DM_DFT_BF16X3_TC05, "bf16x3_tcgen05")):
        for _ in range(args.warmup):
            dm.dm_dft2(frames, work=work, out=out, precision=prec)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            dm.dm_dft2(frames, work=work, out=out, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / args.steps
        if prec == dm.DM_DFT_BF16X3_TC05:
            dm.dm_dft2_check()   # no bounded wait gave up
        got = out[sample].cpu().numpy().astype(np.complex128)
        err = float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))
        res[name] = {"frames_per_s": nf / sec, "ms_per_batch": 1e3 * sec, "rel_l2_vs_fp64": err,
                     "hbm_gbs": nf * s.n * s.n * 32 / sec / 1e9}
    # tensor-core work: the mma.sync form takes 4 radix-16 stages, each 12
    # m16n8k16 products per 8 lines of 16 points; the tcgen05 form 2 passes of
    # 256 rows, each 3 products of (1 x 512) by (512 x 512) real matrices
    flops_mma = nf * s.n * s.n * 4 * (12 * 2 * 16 * 8 * 16) / (8 * 16)
    flops_tc05 = nf * 2 * s.n * 3 * 2 * (2 * s.n) * (2 * s.n)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        bf16_peak = 1900.0
    for name, fl in (("bf16x3_tensor", flops_mma), ("bf16x3_tcgen05", flops_tc05)):
        res[name]["tensor_tflops"] = fl / (res[name]["ms_per_batch"] / 1e3) / 1e12
        res[name]["tensor_frac_of_measured_bf16"] = res[name]["tensor_tflops"] / bf16_peak
    tc = res["bf16x3_tcgen05"]
    tflops = tc["tensor_tflops"]
    if rank == 0:
        print(json.dumps({
            "metric": "frames/s, batched 256x256 2-D DFT", "value": tc["frames_per_s"], "unit": "frames/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "bf16x3 (split operands, fp32 accumulation)", "data": "synthetic",
            "config": {"workload": f"exit waves of the first {views} views of {WORKLOAD} ({nf} frames)",
                       "error_sample_frames": int(sample.numel())},
            "forms": res,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": tflops / bf16_peak, "peak_kind": "measured bf16 (MEASURED_PEAKS.json, burst)",
                         "flops_per_batch": flops_tc05,
                         "kernel": "k_dft256_rows_tc05 (tcgen05.mma kind::f16, bf16 hi/lo, TMEM accumulators)"},
        }), flush=True)


TRAIN_SCANS = 20        # DM-refined training data: 20 scans x 2,500 views = 50,000 frames
TRAIN_SEED = 5000
FRESH_SEED = 9000       # two further scans, never trained on


def trained_warm_net(steps):
    """The warm-start network trained as the learned-start configuration
    states: 6 levels, 1.96 M parameters, 50,000 frames of 20 simulated 4-mode
    scans with targets refined by 20 DM iterations, the phase-gauge-invariant
    loss, ``steps`` Adam steps of 64.  Returns (net, record)."""
    import torch
    from paper_1808_10375_gb300 import dm, warmstart
    t0 = time.perf_counter()
    x, t, _ = warmstart.refined_pairs(TRAIN_SCANS, TRAIN_SEED, dm_iters=20)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = dm.dm_net_create(max_batch=64, seed=11)
    dm.dm_net_set_loss(net, dm.DM_NET_LOSS_GAUGE)
    t0 = time.perf_counter()
    losses = warmstart.train(net, steps=steps, batch=64, lr=1e-3, seed=12, data=(x, t))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, t
    xf, tf, gf = warmstart.refined_pairs(2, FRESH_SEED, dm_iters=20)
    rec = {"frames": TRAIN_SCANS * 2500, "scans": TRAIN_SCANS, "targets": "refined by 20 DM iterations",
           "loss": "phase-gauge invariant", "params": dm.dm_net_param_count(net), "steps": steps,
           "data_s": t_data, "train_s": t_train, "samples_per_s": steps * 64 / t_train,
           "loss_first": losses[0][1], "loss_last": losses[-1][1],
           "fresh_scans": {"frames": int(xf.shape[0]),
                           "fit_to_dm_refined_targets": warmstart.fit(net, xf, tf),
                           "fit_to_true_object": warmstart.fit(net, xf, gf),
                           "dm_refined_target_vs_true_object": warmstart.fit_of(tf, gf)}}
    del xf, tf, gf
    torch.cuda.empty_cache()
    return net, rec


def run_warmstart(args, rank, local):
    """The learned warm start: train the encoder-decoder (the library's BF16
    kernels) on 50,000 DM-refined frames, measure its fit on the frames of two
    fresh scans, stitch its start for a 4-mode 128x128 scan (12x12 views,
    noise-free) and run DM from it and from the flat start; DM's Fourier
    error after --judge-iters trial iterations picks the start."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm, warmstart
    from synth import make_scan
    from synth import warmstart as ws
    torch.cuda.set_device(local)
    steps = args.steps if args.steps != 30 else 3000
    net, training = trained_warm_net(steps)
    cfg = dict(n=128, modes=4, grid=(12, 12), step=10, jitter=1, obj=(250, 250), probe="hg", fwhm=ws.FWHM,
               photons=ws.PHOTONS, seed=13)
    scan = make_scan(cfg, noise=False)
    o_warm = warmstart.predict_start(net, scan.intensities, scan.pos, scan.obj_shape)
    _, pick, ef = warmstart.judged_start(scan, scan.probe, o_warm, trial_iters=args.judge_iters)
    res = warmstart.compare(scan, scan.probe, o_warm, iters=200)
    levels = (0.2, 0.1, 0.05, 0.02, 0.01, 1e-3)
    runs = {name: {"start_error": r["errors"][0][1], "final_error": r["errors"][-1][1], "wall_s": r["wall_s"],
                   "iterations_to": {str(lv): warmstart.iterations_to(r["errors"], lv) for lv in levels}}
            for name, r in res.items()}
    nparams = dm.dm_net_param_count(net)
    dm.dm_net_free(net)
    if rank == 0:
        print(json.dumps({
            "metric": "DM iterations to object error, learned warm start vs flat start", "value": runs["warm"]["final_error"],
            "unit": "relative L2 object error after 200 iterations", "higher_is_better": False, "n_gpus": 1,
            "dtype": "bf16 weights, fp32 accumulation", "data": "synthetic",
            "config": {"workload": "warm-start network: 1x128x128 diffraction amplitude -> 2x64x64 object patch, "
                                   f"{steps} Adam steps of 64 on 50,000 DM-refined frames; judged on a noise-free "
                                   "4-mode 128x128 scan, 12x12 views at 10 px, 250x250 object",
                       "params": nparams},
            "training": training, "judge": {"pick": pick, "trial_iterations": args.judge_iters,
                                            "fourier_error_after_trial": ef}, "runs": runs,
        }), flush=True)


def run_embed(args, rank, local):
    """The object embedding (Eq. 5 numerator, Sec. III) done inside the
    exit-wave update pass against the same embedding as a pass of its own.

    Fused (dm_iterate): the Fourier-step kernel writes c_j = sum_k conj(P_k)
    psi_j^k for each view while psi_j is still in registers, and the object
    gather only sums c_j.  Separate (dm_run_step Fourier, object, probe): the
    object step first recomputes c_j from the stored exit waves, re-reading
    all of them.  The paper overlaps the embedding of one batch of views with
    the exit-wave update of the next and reports about 20 % from it."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm
    s, p0, o0 = make_inputs(args.views, "cuda")
    n, m, j = s.n, s.modes, s.views
    h, w = s.obj_shape
    params = dm.dm_params_default(n=n, modes=m, views=j, obj_h=h, obj_w=w, beta=0.8)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = dm.dm_init(params, dev(s.pos), s.intensities, dev(p0), dev(o0), stream=stream.cuda_stream)

    def separate(k):
        for _ in range(k):
            dm.dm_run_step(ctx, dm.DM_STEP_FOURIER)
            dm.dm_run_step(ctx, dm.DM_STEP_OBJECT)
            dm.dm_run_step(ctx, dm.DM_STEP_PROBE)

    def timed(fn):
        fn(args.warmup)
        torch.cuda.synchronize()
        dm.dm_set_timing(ctx, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        kt = {dm.dm_kernel_name(k): dm.dm_get_timing(ctx, k) for k in range(dm.DM_KERNEL_COUNT)}
        dm.dm_set_timing(ctx, False)
        per = {k: v[0] / v[1] for k, v in kt.items() if v[1]}
        return e0.elapsed_time(e1) / args.steps, per

    with ClockSampler(gpu_index(local)) as clk:
        fused_ms, fused_k = timed(lambda k: dm.dm_iterate(ctx, k))
        sep_ms, sep_k = timed(separate)
    dm.dm_free(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": j * m / (fused_ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fused_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": ("embed: " + WORKLOAD_DESC if args.views is None
                                    else f"embed: {WORKLOAD_DESC} (first {j} views)"),
                       "l2": "inputs larger than L2"},
            "fused": {"ms_per_iteration": fused_ms, "kernels_ms": fused_k},
            "separate": {"ms_per_iteration": sep_ms, "kernels_ms": sep_k,
                         "value": j * m / (sep_ms / 1e3)},
            "fused_speedup": sep_ms / fused_ms,
            "gpu_launches": KERNELS_PER_ITER * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_tte(args, rank, local):
    """Time to object error 1e-3 on the 4-mode 128x128 scan (2,500 views at
    10 px, 640x640 object), simulated without noise so that the reference is
    the true object: plain FP32 DM against the mixed-precision form
    (complex-half exit waves, back to complex64 once the Eq. 6 object change
    drops below --tte-psi-switch).

    Error: relative L2 of the object after the best complex scalar, on the
    pixels where sum_j sum_k |P_k|^2 reaches 0.1 of its maximum.  The probe
    is the true one and stays fixed: with the probe free, a linear phase ramp
    moved from the object to the probe changes no intensity, so the object
    would be fixed only up to that ramp.  Starts: a random object (white
    amplitude in [0.5, 1] and phase in [-pi/2, pi/2], three seeds), the flat
    object, and the judged warm start (the network trained here, stitched,
    with DM's Fourier error after --judge-iters trial iterations choosing between it and
    the flat start).  Runs: FP32 from each start, the mixed form from the
    random starts and the judged start.  Device seconds are CUDA-event time of the
    iterations (for the mixed form including its per-iteration check of the
    switch); the object is copied back and scored every 10 iterations
    outside it."""
    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm, warmstart
    from synth import make_scan
    from synth import warmstart as ws
    scan = make_scan("mm128", noise=False)
    n, m, j = scan.n, scan.modes, scan.views
    h, w = scan.obj_shape
    den = np.zeros((h, w))
    p2 = np.sum(np.abs(scan.probe) ** 2, axis=0)
    for r, c in scan.pos:
        den[r:r + n, c:c + n] += p2
    covered = den >= 0.1 * den.max()
    starts = {"flat": np.ones((h, w), np.complex64)}
    for k, seed in enumerate((2002, 2003, 2004)):
        rng = np.random.Generator(np.random.PCG64(seed))
        starts["random" if k == 0 else f"random{k}"] = ((0.5 + 0.5 * rng.random((h, w))) * np.exp(
            1j * np.pi * (rng.random((h, w)) - 0.5))).astype(np.complex64)
    train_info = None
    starts["judged"] = starts["flat"]
    if args.tte_train_steps > 0:
        net, training = trained_warm_net(args.tte_train_steps)
        t_train = training["data_s"] + training["train_s"]
        t0 = time.perf_counter()
        o_warm = warmstart.predict_start(net, scan.intensities, scan.pos, scan.obj_shape)
        chosen, pick, ef = warmstart.judged_start(scan, scan.probe, o_warm, trial_iters=args.judge_iters)
        t_pick = time.perf_counter() - t0
        dm.dm_net_free(net)
        starts["judged"] = chosen
        train_info = {"steps": args.tte_train_steps, "train_s": t_train, "training": training,
                      "predict_and_judge_s": t_pick,
                      "judge_pick": pick, "judge_trial_iterations": args.judge_iters,
                      "fourier_error_after_trial": ef,
                      "predicted_start_error": ws.object_error(o_warm.detach().cpu().numpy(), scan.obj, covered)}
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    levels = (1e-1, 1e-2, 1e-3)
    block = 10
    arms = [("fp32_random", "random", dm.DM_PSI_FP32), ("fp32_flat", "flat", dm.DM_PSI_FP32),
            ("fp32_judged", "judged", dm.DM_PSI_FP32), ("mixed_random", "random", dm.DM_PSI_FP16),
            ("mixed_judged", "judged", dm.DM_PSI_FP16)]
    for k in (1, 2):   # two more random starts in both forms: the spread of the slow phase
        arms += [(f"fp32_random{k}", f"random{k}", dm.DM_PSI_FP32), (f"mixed_random{k}", f"random{k}", dm.DM_PSI_FP16)]
    runs = {}
    with ClockSampler(gpu_index(local)) as clk:
        for name, start, prec in arms:
            o0 = starts[start]
            params = dm.dm_params_default(n=n, modes=m, views=j, obj_h=h, obj_w=w, beta=0.8,
                                          probe_update_start=1 << 30, psi_precision=prec,
                                          psi_switch=args.tte_psi_switch if prec == dm.DM_PSI_FP16 else 0.0)
            ctx = dm.dm_init(params, scan.pos, scan.intensities, scan.probe.astype(np.complex64), o0,
                             stream=stream.cuda_stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            dev_s, it, err = 0.0, 0, ws.object_error(o0, scan.obj, covered)
            first = {}
            start_err = err
            t0 = time.perf_counter()
            while it < args.tte_iters:
                e0.record(stream)
                dm.dm_iterate(ctx, block)
                e1.record(stream)
                o = dm.dm_get_object(ctx)
                dev_s += e0.elapsed_time(e1) / 1e3
                it += block
                err = ws.object_error(o, scan.obj, covered)
                for lv in levels:
                    if err <= lv and str(lv) not in first:
                        first[str(lv)] = {"iterations": it, "device_s": dev_s, "wall_s": time.perf_counter() - t0}
                if err <= levels[-1]:
                    break
            prec_now, switched_at = dm.dm_get_psi_precision(ctx)
            dm.dm_free(ctx)
            runs[name] = {"start": start, "exit_waves": "complex half, then complex64" if prec else "complex64",
                          "start_error": start_err, "final_error": err, "iterations": it, "device_s": dev_s,
                          "ms_per_iteration": 1e3 * dev_s / max(it, 1), "to": first,
                          "switched_to_complex64_at": switched_at if prec else None}
    # the FP64 oracle per iteration: one process and all host cores, scaled to all views
    from oracle import dm as odm
    cv = 100
    psi = odm.init_exit_waves(scan.probe.astype(np.complex128), starts["flat"].astype(np.complex128), scan.pos[:cv])
    t0 = time.perf_counter()
    odm.dm_iteration(psi, scan.probe.astype(np.complex128), starts["flat"].astype(np.complex128), scan.pos[:cv],
                     scan.intensities[:cv].astype(np.float64), update_probe=False)
    cpu_iter_s = (time.perf_counter() - t0) * j / cv
    nproc, model = host_cpu()
    from oracle.parallel import ProcessDM
    cvn = min(j, 16 * nproc)
    with ProcessDM(np.ascontiguousarray(scan.intensities[:cvn], np.float32), scan.pos[:cvn],
                   scan.probe.astype(np.complex128), starts["flat"].astype(np.complex128), workers=nproc) as pdm:
        t0 = time.perf_counter()
        pdm.iterate()
        cpu_iter_all = (time.perf_counter() - t0) * j / cvn
    base = runs["fp32_random"]["to"].get(str(levels[-1]))
    best = runs["mixed_judged"]["to"].get(str(levels[-1]))
    if rank == 0:
        print(json.dumps({
            "metric": "time to object error 1e-3: warm-started mixed-precision form vs plain FP32 DM from a random start",
            "unit": "s", "value": best["device_s"] if best else None, "higher_is_better": False, "n_gpus": 1,
            "fp32_random_s": base["device_s"] if base else None,
            "speedup_vs_fp32_random": (base["device_s"] / best["device_s"]) if base and best else None,
            "dtype": "f32 arithmetic; mixed form: exit waves stored as f16 until the switch",
            "data": "synthetic", "psi_switch": args.tte_psi_switch,
            "config": {"workload": "tte: 4-mode difference map, 128x128 frames, 50x50 scan (2,500 views) at 10 px, "
                                   "640x640 object, noise-free, true probe held fixed, beta 0.8",
                       "error": "relative L2 after the best complex scalar on pixels with sum |P|^2 >= 0.1 max"},
            "runs": runs, "learned": train_info, "clocks": clk.summary(),
            "cpu_baseline": {"kind": "oracle", "cores": nproc, "s_per_iteration": cpu_iter_all,
                             "sample": f"one FP64 oracle iteration over the first {cvn} views with the views split "
                                       f"over {nproc} processes, scaled to {j}",
                             "one_core_s_per_iteration": cpu_iter_s, "cpu_model": model},
        }), flush=True)


def make_scan_cfg(cfg):
    from synth import make_scan
    return make_scan(cfg, backend="torch", device="cuda")


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch16":
        run_batch16(args, rank, local)
        return
    if args.workload == "dft256":
        run_dft256(args, rank, local)
        return
    if args.workload == "warmstart":
        run_warmstart(args, rank, local)
        return
    if args.workload == "embed":
        run_embed(args, rank, local)
        return
    if args.workload == "tte":
        run_tte(args, rank, local)
        return
    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        pg = tdist

    barrier, max_over_ranks = rank_collectives(pg, "cuda")

    import __graft_entry__
    __graft_entry__.build()
    from paper_1808_10375_gb300 import dm

    wname = args.workload if args.workload in WORKLOADS else WORKLOAD
    wdesc = WORKLOADS[wname]
    s, p0, o0 = make_inputs(args.views, "cuda", wname)
    n, m, j = s.n, s.modes, s.views
    h, w = s.obj_shape
    params = dm.dm_params_default(n=n, modes=m, views=j, obj_h=h, obj_w=w, beta=0.8,
                                  psi_precision=dm.DM_PSI_FP16 if args.psi == "fp16" else dm.DM_PSI_FP32)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()          # the library's stream: every kernel and event below
    torch.cuda.set_stream(stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = dm.dm_init(params, dev(s.pos), s.intensities, dev(p0), dev(o0), stream=stream.cuda_stream)
    form_req = {"strip": dm.DM_FOURIER_STRIP, "split": dm.DM_FOURIER_SPLIT,
                "cluster": dm.DM_FOURIER_CLUSTER}.get(args.form)
    if form_req is not None:
        dm.dm_set_fourier_form(ctx, form_req)
    if args.autotune > 0:
        dm.dm_autotune(ctx, sample_views=min(j, args.autotune))
    form = {dm.DM_FOURIER_SPLIT: "split", dm.DM_FOURIER_CLUSTER: "cluster"}.get(dm.dm_get_fourier_form(ctx), "strip")
    plan = dm.dm_get_plan(ctx)
    # iterations replay captured CUDA graphs (one per pair of current object and
    # probe buffers, captured during the warm-up)
    dm.dm_set_graph(ctx, True)
    dm.dm_iterate(ctx, max(args.warmup, 2))
    dm.dm_sync(ctx)

    # ---- device-timed region -------------------------------------------------
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index(local)) as clk:
        e0.record(stream)
        dm.dm_iterate(ctx, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    t_ms = max_over_ranks(e0.elapsed_time(e1))
    # per-kernel times (CUDA events around every launch, which runs the
    # iterations kernel by kernel): a second pass of the same iterations
    dm.dm_set_timing(ctx, True)
    dm.dm_iterate(ctx, args.steps)
    dm.dm_sync(ctx)
    kt = {dm.dm_kernel_name(k): dm.dm_get_timing(ctx, k) for k in range(dm.DM_KERNEL_COUNT)}
    dm.dm_set_timing(ctx, False)
    eps_obj, eps_probe, ferr = dm.dm_get_error(ctx)
    dm.dm_free(ctx)
    value = job_throughput(world, j, m, args.steps, t_ms / 1e3)

    f_ms, f_n = kt["fourier"]
    hbm, peak_kind = peaks()
    psi_bytes = 4 if args.psi == "fp16" else 8
    f_bytes = fourier_bytes_per_view(n, m, psi_bytes) * j
    c_bytes = object_source_bytes_per_view(n) * j
    launch_s = f_ms / f_n / 1e3 if f_n else None
    achieved = f_bytes / launch_s / 1e9 if f_n else None
    fp32_peak = dm.dm_fp32_peak()
    fft_tflops = fourier_flops_per_view(n, m) * j / launch_s / 1e12 if f_n else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None,
                "traffic": stored_traffic(j, form) if (wname == WORKLOAD and args.psi == "fp32") else None,
                "kernel": FORM_KERNEL_NAME[form],
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": f_bytes, "avg_launch_ms": f_ms / f_n if f_n else None,
                "object_source_bytes_per_launch": c_bytes,
                "frac_with_object_source": ((f_bytes + c_bytes) / launch_s / 1e9 / hbm) if f_n else None,
                "fp32_pipe": {"achieved": fft_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                              "frac": (fft_tflops / fp32_peak) if fft_tflops else None,
                              "flops_per_launch": fourier_flops_per_view(n, m) * j,
                              "peak_kind": "measured (dm_fp32_peak, FMA = 2)",
                              "count": "5 L log2 L per complex transform of L = N^2 points, forward and "
                                       "inverse, every view and mode"}}
    iter_bytes = iteration_bytes_per_view(n, m, psi_bytes) * j
    breakdown = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else None, "launches": v[1],
                     "share": v[0] / max(1e-9, sum(x[0] for x in kt.values()))} for k, v in kt.items()}

    # ---- end to end through the C ABI with host buffers ---------------------
    e2e = None
    if not args.no_e2e:
        inten_h = torch.empty(s.intensities.shape, dtype=torch.float32, pin_memory=True)
        inten_h.copy_(s.intensities)
        pos_h = torch.from_numpy(np.ascontiguousarray(s.pos)).pin_memory()
        p0_h = torch.from_numpy(p0).pin_memory()
        o0_h = torch.from_numpy(o0).pin_memory()
        o_out = torch.empty((h, w), dtype=torch.complex64, pin_memory=True)
        p_out = torch.empty((m, n, n), dtype=torch.complex64, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = dm.dm_init(params, pos_h, inten_h, p0_h, o0_h, stream=stream.cuda_stream)
        if form_req is not None:
            dm.dm_set_fourier_form(c2, form_req)
        dm.dm_set_graph(c2, True)   # as in the device-timed loop (the captures happen in this session)
        dm.dm_iterate(c2, args.steps)
        dm.dm_get_object(c2, out=o_out)
        dm.dm_get_probe(c2, out=p_out)
        dm.dm_get_error(c2)
        t1 = time.perf_counter()
        dm.dm_free(c2)
        barrier()
        e2e_s = max_over_ranks(t1 - t0)
        h2d = inten_h.numel() * 4 + pos_h.numel() * 4 + p0_h.numel() * 8 + o0_h.numel() * 8
        d2h = o_out.numel() * 8 + p_out.numel() * 8 + 8 * (2 + m)
        e2e = {"value": job_throughput(world, j, m, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "session": f"dm_init from pinned host buffers + {args.steps} iterations (CUDA-graph replay, "
                          f"captured in the session) + object, probe and metrics to host, per step = session / "
                          f"{args.steps}",
               "fourier_plan": "default"}

    # ---- CPU oracle baseline (rank 0, N = 1) ---------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_line(s, p0, o0, j, m, args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.psi == "fp32" else "f32 arithmetic, exit waves stored as f16", "data": "synthetic",
            "config": {"workload": wdesc if args.views is None else f"{wdesc} (first {j} views)",
                       "n": n, "modes": m, "views": j, "object": [h, w], "beta": 0.8,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (exit waves %.1f GB)" % (j * m * n * n * 8 / 1e9),
                       "fourier_plan": dict(plan, autotuned=args.autotune > 0),
                       "fourier_form": form,
                       "launch": "CUDA-graph replay of each iteration (per-kernel times from a second "
                                 "pass launched kernel by kernel with events)",
                       "iteration_algorithmic_bytes": iter_bytes,
                       "iteration_hbm_frac": iter_bytes / (t_ms / args.steps / 1e3) / 1e9 / hbm},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": KERNELS_PER_ITER * args.steps,
            "clocks": clk.summary(),
            "kernels": breakdown,
            "metrics_last": {"eps_obj": eps_obj, "eps_probe": eps_probe, "fourier_err": ferr},
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
