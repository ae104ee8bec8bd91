"""Throughput and latency of the ELAS path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The JSON line's value is Mpix/s of the plain one-pair path on 640x480 pairs
with 256 disparities: one pair per step, the whole path on the GPU
(descriptors, support points, triangulation, plane prior, dense matching,
LR check, post-processing), inputs resident in HBM, L2 flushed before every
step.  The same line carries:
  e2e          the same metric through the host-buffer call (copies timed);
  roofline     the dense argmin kernel (one launch covers both reference
               images) against its binding roof (HBM bytes or the measured
               SAD16 ceiling, whichever bounds the launch from below), both
               shown, timed by events inside the timed steps;
  batch        64 pairs of 1242x375 with 256 disparities in one batched wave
               (one launch per kernel for all pairs, CUDA graph, tuned tile
               shapes) against 64 runs of the plain path, with the batched
               dense kernel's roofline;
  batch_census the same batch with the paper's census variant (9x9
               support and 5x5 dense census windows, Hamming costs);
  mixed_batch  128 pairs of mixed sizes and disparity ranges in one wave
               against 128 plain runs;
  serving      8 simulated cameras with Poisson arrivals (600 pairs/s in
               total, 60 s): the continuous-batching server against the
               plain per-pair loop, p50/p99 latency and pairs/s;
  serving_saturated  the same cameras at 4000 pairs/s offered (above the
               plain path's rate): served pairs/s and latency of both;
  cpu_baseline the oracle on the host cores;
  summary      the figures of every section, last on the line.
N > 1 runs N independent replicas, one per GPU (pairs are independent; no
collective on the data path); the extra sections run on rank 0.
``--impl reference`` times the CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1802_07210_gb300 import synth  # noqa: E402

METRIC = "Mpix/s & pairs/s at 640x480 D=256; p50/p99 served latency vs per-pair path"
WORKLOADS = {"vga_640": (synth.VGA_640, 2), "small_320": (synth.SMALL_320, 1),
             "kitti_1242": (synth.KITTI_1242, 3)}
# kernels of one plain step: descriptors 1; support 4 (match, consistency,
# redundancy + grids, compaction); triangulation 10 (init, points, cell scan,
# scatter, dedup, group pass, CTA pass, triangle scan, emit, emit big); plane
# prior 3 (setup, extra-unit list, draw); dense 1; LR 1; post-processing 1
# (fused) or 0.  No memsets.
KERNELS_PER_STEP = {True: 21, False: 20}
STAGES = ("descriptors", "support", "triangulation", "plane_prior", "dense_argmin", "lr_post")
# bytes a dense launch must move at least: both descriptor images read once
# (32 B/px), the two prior maps read (4 B/px), the two maps written (4 B/px)
DENSE_MIN_BYTES_PER_PX = 40


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_warm(_):
    """Loads the oracle in a worker before any step is timed."""
    import oracle
    oracle.lib()
    return os.getpid()


def _oracle_pair(args):
    """One pair (rows [0, rows) of it when rows is given) through the oracle:
    a worker of the all-cores runs."""
    name, idx, cfg = args[:3]
    rows = args[3] if len(args) > 3 else None
    import oracle
    wl = {w.name: w for w, _ in WORKLOADS.values()}[name]
    L, R, _ = synth.workload_pair(wl, idx, cfg)
    if rows is not None:
        L, R = np.ascontiguousarray(L[:rows]), np.ascontiguousarray(R[:rows])
    t0 = time.perf_counter()
    oracle.pipeline(L, R, wl.params, postprocess_on=wl.postprocess)
    return time.perf_counter() - t0


def cpu_baseline(wl, cfg, seconds=12.0):
    """The oracle as it stands on whole pairs of the workload: one core for
    about `seconds` of CPU work, then four pairs per core on every core at
    once (independent processes, started with spawn)."""
    import multiprocessing as mp
    import oracle
    oracle.lib()
    n, t = 0, 0.0
    while t < seconds or n == 0:
        L, R, _ = synth.workload_pair(wl, 100 + n, cfg)
        t0 = time.perf_counter()
        oracle.pipeline(L, R, wl.params, postprocess_on=wl.postprocess)
        t += time.perf_counter() - t0
        n += 1
        if n >= 48:
            break
    px = wl.spec.w * wl.spec.h
    one = {"value": n * px / t / 1e6, "unit": "Mpix/s", "cores": 1, "pairs_per_s": n / t,
           "sample": "%d whole %dx%d pairs through the oracle pipeline (%.1f s)" % (n, wl.spec.w, wl.spec.h, t)}
    cores = host_cores()
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_warm, range(cores))
            per = 4  # pairs per core: about 20 s of CPU work at 640x480
            t0 = time.perf_counter()
            pool.map(_oracle_pair, [(wl.name, 300 + i, cfg) for i in range(per * cores)], chunksize=per)
            wall = time.perf_counter() - t0
        allc = {"value": per * cores * px / wall / 1e6, "cores": cores, "pairs_per_s": per * cores / wall,
                "sample": "%d whole %dx%d pairs, %d per core on %d cores at once (%.1f s wall)" % (
                    per * cores, wl.spec.w, wl.spec.h, per, cores, wall)}
    except Exception as e:  # the single-core number stands alone
        allc = {"error": str(e)}
    if "value" in allc:
        return {"value": allc["value"], "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                "sample": allc["sample"], "pairs_per_s": allc["pairs_per_s"], "one_core": one}
    return dict(one, kind="oracle", all_cores=allc)


def run_reference(args, wl, cfg, budget_s=200.0):
    """The oracle on the host cores: every step runs one pair per core, all at
    once in spawned worker processes, and takes its wall time. The first
    warm-up step runs whole pairs; when whole pairs would take the run past
    about `budget_s`, the later steps run the top band of rows of each pair
    (the same images and parameters, fewer rows), sized to fit. The oracle's
    cost per pixel falls with fewer rows, so a band overstates its rate."""
    import multiprocessing as mp
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.lib()
    cores = host_cores()
    h = wl.spec.h
    rows, ms = h, []
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_warm, range(cores))
        for i in range(args.warmup + args.steps):
            jobs = [(wl.name, 1000 * (i % 4) + c, cfg, rows) for c in range(cores)]
            t0 = time.perf_counter()
            pool.map(_oracle_pair, jobs)
            dt = time.perf_counter() - t0
            if i == 0:
                per_step = budget_s / max(1, args.warmup + args.steps - 1)
                rows = int(min(h, max(16, h * per_step / dt)))
            if i >= args.warmup:
                ms.append(1e3 * dt)
    t = sum(ms) / 1e3
    px = wl.spec.w * rows
    val = args.steps * cores * px / t / 1e6
    sample = "%d steps of %d pairs (one per core, spawned workers), each the top %d of %d rows of a %s pair" % (
        args.steps, cores, rows, h, wl.name)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": wl.name, "w": wl.spec.w, "h": wl.spec.h,
                                            "disp_max": wl.disp_max, "pairs_per_step": cores,
                                            "rows_per_pair": rows, "sample": sample},
            "pairs_per_s": args.steps * cores * rows / h / t,
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(torch, dist, ws, value, device):
    """The largest of every rank's value (a time): the job is as slow as its
    slowest replica."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, steps, units_per_step, total_ms):
    """Whole-job rate of ws independent replicas that each did `steps` steps
    of `units_per_step` units, the slowest in total_ms."""
    return ws * steps * units_per_step / (total_ms / 1e3)


def replica_seed(rank, i):
    """Pair seeds of a replica: disjoint across ranks."""
    return rank * 1000 + i


def _timed(torch, stream, flush, fn, steps):
    """Device ms of each of `steps` calls of fn(i), L2 flushed before each."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        fn(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def pair_dense_evals(B, torch, wl, L, R, dev):
    """Algorithmic candidate evaluations of the dense step for one pair (the
    intermediates come from the library's own calls; host triangulation)."""
    prm = B.as_params(wl.params)
    tL, tR = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
    descL, descR = B.elas_descriptors(tL, tR)
    sp = B.elas_support_points(descL, descR, prm)
    torch.cuda.synchronize()
    n = int(sp["count"].item())
    lst_h = sp["list"][:n].cpu().numpy()
    triL = torch.from_numpy(B.elas_triangulate(lst_h, False)).to(dev)
    triR = torch.from_numpy(B.elas_triangulate(lst_h, True)).to(dev)
    lst = sp["list"][:max(n, 1)].contiguous()
    h, w = L.shape
    dpL = B.elas_plane_prior(lst, triL, w, h, prm, False)
    dpR = B.elas_plane_prior(lst, triR, w, h, prm, True)
    work = dict(descL=descL.cpu().numpy(), descR=descR.cpu().numpy(), dpL=dpL.cpu().numpy(),
                dpR=dpR.cpu().numpy(), gridL=sp["grid_L"].cpu().numpy(), gridR=sp["grid_R"].cpu().numpy())
    return dense_work(work, prm, w, h)


def run_batch_section(B, torch, dev, stream, flush, steps, npairs, distinct, peak_gsad, hbm, tune=True,
                      overrides=None):
    """64 x 1242x375 D=256 through one batched wave vs the plain path
    (overrides: parameters of the paper's variant, without the dense
    roofline)."""
    wl, cfg = synth.KITTI_1242, 3
    if overrides:
        wl = synth.Workload(wl.name, wl.spec, wl.disp_max, wl.postprocess, dict(wl.params, **overrides))
    w, h = wl.spec.w, wl.spec.h
    pool = [synth.workload_pair(wl, 500 + i, cfg)[:2] for i in range(distinct)]
    imgL = [torch.from_numpy(pool[i % distinct][0]).to(dev) for i in range(npairs)]
    imgR = [torch.from_numpy(pool[i % distinct][1]).to(dev) for i in range(npairs)]
    dL = [torch.empty((h, w), dtype=torch.int16, device=dev) for _ in range(npairs)]
    dR = [torch.empty_like(t) for t in dL]
    b = B.Batch([(w, h)] * npairs, wl.params)
    tuned = b.tune(imgL, imgR, dL) if tune else b.config()
    for _ in range(3):
        b.run(imgL, imgR, dL, dR)
    ms = _timed(torch, stream, flush, lambda i: b.run(imgL, imgR, dL, dR), steps)
    prof = [b.profile() for _ in range(3)]
    stage = {k: float(np.median([p[k] for p in prof])) for k in prof[0]}
    nsup = b.stats()["n_support"]
    b.close()
    pl = B.Pipeline(w, h, wl.params)
    for i in range(npairs):
        pl.run(imgL[i], imgR[i], dL[i], dR[i])
    ms_plain = _timed(torch, stream, flush, lambda i: [pl.run(imgL[k], imgR[k], dL[k], dR[k]) for k in range(npairs)],
                      max(3, steps // 3))
    pl.close()
    t_b, t_p = float(np.mean(ms)), float(np.mean(ms_plain))
    if overrides:
        return {"workload": "%d x %s" % (npairs, wl.name), "parameters": overrides, "pairs": npairs,
                "distinct_pairs": distinct, "ms_per_batch": t_b, "pairs_per_s": npairs / (t_b * 1e-3),
                "mpix_per_s": npairs * w * h / (t_b * 1e-3) / 1e6, "plain_ms_per_batch": t_p,
                "plain_pairs_per_s": npairs / (t_p * 1e-3), "speedup_vs_plain": t_p / t_b, "tuned": tuned,
                "stages_ms": stage, "support_points_first": nsup[:4], "l2": "flushed before every timed batch"}
    evals = sum(pair_dense_evals(B, torch, wl, L, R, dev) for L, R in pool) * (npairs // distinct)
    evals += sum(pair_dense_evals(B, torch, wl, *pool[i], dev) for i in range(npairs % distinct))
    roof = {"kernel": "cell_kernel_b (dense argmin, every pair and both reference images in one launch)"}
    roof.update(dense_roofline(evals, DENSE_MIN_BYTES_PER_PX * w * h * npairs, stage["dense_argmin"], peak_gsad,
                               hbm[0], hbm[1]))
    roof["time_source"] = "CUDA events around the launch in an eager run of the same batch"
    return {"workload": "%d x %s" % (npairs, wl.name), "pairs": npairs, "distinct_pairs": distinct,
            "ms_per_batch": t_b, "pairs_per_s": npairs / (t_b * 1e-3), "mpix_per_s": npairs * w * h / (t_b * 1e-3) / 1e6,
            "plain_ms_per_batch": t_p, "plain_pairs_per_s": npairs / (t_p * 1e-3),
            "speedup_vs_plain": t_p / t_b, "tuned": tuned, "stages_ms": stage, "support_points_first": nsup[:4],
            "launches_per_batch": 21, "graph": True,
            "l2": "flushed before every timed batch", "roofline_dense": roof}


def run_mixed_section(B, torch, dev, stream, flush, steps, npairs, tune=True):
    """128 pairs of mixed sizes and disparity ranges: one wave vs plain runs."""
    spec = synth.mixed_batch(npairs, 4)
    distinct = {}
    for wl, _ in spec:
        distinct.setdefault(wl.name, wl)
    pool = {name: synth.workload_pair(wl, 700, 4)[:2] for name, wl in distinct.items()}
    imgL = [torch.from_numpy(pool[wl.name][0]).to(dev) for wl, _ in spec]
    imgR = [torch.from_numpy(pool[wl.name][1]).to(dev) for wl, _ in spec]
    dL = [torch.empty(t.shape, dtype=torch.int16, device=dev) for t in imgL]
    dR = [torch.empty_like(t) for t in dL]
    shapes = [(wl.spec.w, wl.spec.h) for wl, _ in spec]
    b = B.Batch(shapes, [wl.params for wl, _ in spec])
    tuned = b.tune(imgL, imgR, dL) if tune else b.config()
    for _ in range(3):
        b.run(imgL, imgR, dL, dR)
    ms = _timed(torch, stream, flush, lambda i: b.run(imgL, imgR, dL, dR), steps)
    b.close()
    pls = {name: B.Pipeline(wl.spec.w, wl.spec.h, wl.params) for name, wl in distinct.items()}
    names = [wl.name for wl, _ in spec]

    def plain(_):
        for k in range(npairs):
            pls[names[k]].run(imgL[k], imgR[k], dL[k], dR[k])
    plain(0)
    ms_plain = _timed(torch, stream, flush, plain, max(3, steps // 3))
    for p in pls.values():
        p.close()
    px = sum(w * h for w, h in shapes)
    t_b, t_p = float(np.mean(ms)), float(np.mean(ms_plain))
    return {"workload": "%d mixed pairs (sizes %s, D in %s)" % (npairs, synth.MIXED_SIZES, synth.MIXED_D),
            "distinct_pairs": len(pool), "megapixels": px / 1e6, "ms_per_batch": t_b,
            "pairs_per_s": npairs / (t_b * 1e-3), "mpix_per_s": px / (t_b * 1e-3) / 1e6,
            "plain_ms_per_batch": t_p, "plain_pairs_per_s": npairs / (t_p * 1e-3), "speedup_vs_plain": t_p / t_b,
            "tuned": tuned, "l2": "flushed before every timed batch"}


def run_serve_section(B, torch, seconds, rate_per_camera=75.0, seed=5):
    """8 cameras (2 x 640x480 D=128, 4 x 1242x375 D=256, 2 x 1920x1080 D=256),
    Poisson arrivals, host buffers in and out: the continuous-batching server
    against the plain per-pair loop on the same arrival schedule."""
    cams = [synth.scaled_workload(640, 480, 128)] * 2 + [synth.KITTI_1242] * 4 + \
        [synth.scaled_workload(1920, 1080, 256)] * 2
    pool = {}
    for wl in cams:
        if wl.name not in pool:
            pool[wl.name] = [tuple(torch.from_numpy(x).pin_memory() for x in synth.workload_pair(wl, k, 5)[:2])
                             for k in range(2)]
    rng = np.random.default_rng(seed)
    arr = []
    for ci in range(len(cams)):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate_per_camera)
            if t >= seconds:
                break
            arr.append((t, ci))
    arr.sort()

    def run(plain):
        srv = B.Server(plain=plain, lanes=3, max_wave=64)
        ring = {ci: [torch.empty(pool[wl.name][0][0].shape, dtype=torch.int16).pin_memory() for _ in range(256)]
                for ci, wl in enumerate(cams)}
        for ci, wl in enumerate(cams):  # warm-up: creates the slots
            srv.submit(10 ** 9 + ci, pool[wl.name][0][0], pool[wl.name][0][1], ring[ci][0], wl.params)
        got = 0
        while got < len(cams):
            got += len(srv.poll(64, 100))
        lat, done = [], 0
        t0 = time.perf_counter()
        for i, (ta, ci) in enumerate(arr):
            while True:
                now = time.perf_counter() - t0
                if now >= ta:
                    break
                for r in srv.poll(256, 0):
                    lat.append(r["t_done_ms"] - r["t_submit_ms"])
                    done += 1
                if ta - now > 0.0005:
                    time.sleep(min(ta - now - 0.0003, 0.002))
            wl = cams[ci]
            L, R = pool[wl.name][i % 2]
            srv.submit(i, L, R, ring[ci][i % 256], wl.params)
        while done < len(arr):
            for r in srv.poll(256, 200):
                lat.append(r["t_done_ms"] - r["t_submit_ms"])
                done += 1
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array(lat)
        return {"pairs": int(len(lat)), "pairs_per_s": len(lat) / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()), "waves": int(st["waves"]),
                "max_wave": int(st["max_wave_seen"]), "slots": int(st["slots_in_use"]),
                "slot_gb": st["slot_bytes"] / 1e9}

    out = {"cameras": "2x640x480 D=128, 4x1242x375 D=256, 2x1920x1080 D=256",
           "arrivals": "Poisson, %.0f pairs/s per camera, %.0f pairs/s in total, seeded" % (rate_per_camera,
                                                                                          rate_per_camera * len(cams)),
           "offered_pairs_per_s": rate_per_camera * len(cams),
           "seconds": seconds, "requests": len(arr),
           "latency": "submit to outputs on the host (host copies included)",
           "continuous_batching": run(False), "plain_per_pair": run(True)}
    cb, pp = out["continuous_batching"], out["plain_per_pair"]
    out["p50_ratio_plain_over_batched"] = pp["p50_ms"] / cb["p50_ms"]
    out["p99_ratio_plain_over_batched"] = pp["p99_ms"] / cb["p99_ms"]
    return out


def kitti_outliers(d, gt):
    """Accuracy of a disparity map against ground truth with the criterion
    the paper evaluates by: an estimate is an outlier when it differs from
    the truth by at least 3 pixels and by at least 5 %.  Returns the density
    (valid estimates / pixels), the outlier share of the valid estimates and
    the share of all pixels that are invalid or outliers."""
    d = np.asarray(d, np.int64)
    gt = np.asarray(gt, np.int64)
    valid = d >= 0
    err = np.abs(d - gt)
    bad = valid & (err >= 3) & (err >= 0.05 * gt)
    n = d.size
    nv = int(valid.sum())
    return {"density": nv / n, "outliers_of_valid": int(bad.sum()) / max(1, nv),
            "outliers_all": (int(bad.sum()) + n - nv) / n}


def run_accuracy_section(B, torch, dev, npairs=4, steps=(5, 7, 10, 14)):
    """Outlier rates of the LR-checked left map (no post-processing, as the
    paper measures) against the generator's ground truth, for support
    densities set by the candidate lattice step (the support-point count
    falls with the square of the step)."""
    out = {"criterion": "|d - gt| >= 3 and >= 5 % of gt; map: LR-checked left, no post-processing "
                        "(and the same map through the 3x3 median filter, elas_median)",
           "pairs_per_config": npairs}
    for wl, cfg in (WORKLOADS["vga_640"], WORKLOADS["kitti_1242"]):
        h, w = wl.spec.h, wl.spec.w
        pairs = [synth.workload_pair(wl, 200 + i, cfg) for i in range(npairs)]
        rows = {}
        for step in steps:
            prm = dict(wl.params, candidate_stepsize=step)
            pl = B.Pipeline(w, h, prm)
            dL = torch.empty((h, w), dtype=torch.int16, device=dev)
            acc, acc_med, acc_sp, nsup = [], [], [], []
            for L, R, gt in pairs:
                pl.run(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), dL)
                acc.append(kitti_outliers(dL.cpu().numpy(), gt))
                acc_med.append(kitti_outliers(B.elas_median(dL, 1).cpu().numpy(), gt))
                acc_sp.append(kitti_outliers(B.elas_speckle(dL, 1, 200).cpu().numpy(), gt))
                nsup.append(pl.stats()["n_support"])
            pl.close()
            rows["step_%d" % step] = {"support_points": float(np.mean(nsup)),
                                      **{k: float(np.mean([a[k] for a in acc])) for k in acc[0]},
                                      "with_3x3_median": {k: float(np.mean([a[k] for a in acc_med]))
                                                          for k in acc_med[0]},
                                      "with_speckle_1_200": {k: float(np.mean([a[k] for a in acc_sp]))
                                                             for k in acc_sp[0]}}
        # the paper's FPGA-side choices at the default lattice step: the
        # shift-sum threshold and past-only redundancy as flags, and census
        # descriptors with Hamming costs (9x9 / 5x5 as the paper compares,
        # 13x13 / 7x7; with beta 0.1 the plane prior P = [-2, -1, 0] is
        # scaled to Hamming costs of at most 25 instead of [-14, -9, -2])
        variants = {"shift_sum_eq3": dict(flags=8), "past_only_redundancy": dict(flags=16),
                    "both": dict(flags=24),
                    "census_9x9_5x5": dict(census_support_w=9, census_dense_w=5),
                    "census_13x13_7x7": dict(census_support_w=13, census_dense_w=7),
                    "census_9x9_5x5_beta_0.1": dict(census_support_w=9, census_dense_w=5, beta=0.1)}
        var = {}
        for key, ov in variants.items():
            prm = dict(wl.params, **ov)
            pl = B.Pipeline(w, h, prm)
            dL = torch.empty((h, w), dtype=torch.int16, device=dev)
            acc, nsup = [], []
            for L, R, gt in pairs:
                pl.run(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), dL)
                acc.append(kitti_outliers(dL.cpu().numpy(), gt))
                nsup.append(pl.stats()["n_support"])
            pl.close()
            var[key] = {"support_points": float(np.mean(nsup)),
                        **{k: float(np.mean([a_[k] for a_ in acc])) for k in acc[0]}}
        rows["step_5_variants"] = var
        # the paper's down-sampling (Sec. VII): support extracted at every
        # pixel, then 1/k of the filtered points kept
        down = {}
        for k in (8, 14, 32):
            prm = dict(wl.params, candidate_stepsize=1, support_downsample=k)
            pl = B.Pipeline(w, h, prm)
            dL = torch.empty((h, w), dtype=torch.int16, device=dev)
            acc, nsup = [], []
            for L, R, gt in pairs:
                pl.run(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), dL)
                acc.append(kitti_outliers(dL.cpu().numpy(), gt))
                nsup.append(pl.stats()["n_support"])
            pl.close()
            down["1_of_%d" % k] = {"support_points": float(np.mean(nsup)),
                                   **{k_: float(np.mean([a_[k_] for a_ in acc])) for k_ in acc[0]}}
        rows["every_pixel_downsampled"] = down
        out[wl.name] = rows
    # the median kernel alone on a 1242x375 map (inputs resident; radius 1
    # and 2), against the measured copy bandwidth at its minimum bytes
    hbm_gbs, _ = _peaks()
    wl = WORKLOADS["kitti_1242"][0]
    h, w = wl.spec.h, wl.spec.w
    d = torch.randint(-1, 250, (h, w), dtype=torch.int16, device=dev)
    o = torch.empty_like(d)
    timing = {}
    for r in (1, 2):
        for _ in range(3):
            B.elas_median(d, r, o)
        torch.cuda.synchronize()
        # 20 launches in a CUDA graph, so that host launch latency stays out
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for _ in range(20):
                    B.elas_median(d, r, o)
        torch.cuda.current_stream().wait_stream(side)
        g.replay()
        torch.cuda.synchronize()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record()
        g.replay()
        b_.record()
        b_.synchronize()
        us = a_.elapsed_time(b_) * 1e3 / 20
        gbs = 4.0 * w * h / (us * 1e-6) / 1e9  # 2 B read + 2 B written per pixel
        timing["radius_%d" % r] = {"us": us, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm_gbs}
    out["median_kernel_1242x375"] = timing
    out["speckle"] = speckle_timing(B, torch, dev, hbm_gbs)
    out["census_640x480"] = census_timing(B, torch, dev, hbm_gbs)
    return out


def _graph_us(torch, fn, n=20):
    """Mean time of fn() over n launches replayed from one CUDA graph (host
    launch latency left out), after warm-up."""
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for _ in range(n):
                fn()
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_.record()
    g.replay()
    b_.record()
    b_.synchronize()
    return a_.elapsed_time(b_) * 1e3 / n


def speckle_timing(B, torch, dev, hbm_gbs):
    """Small-segment removal (threshold 1, 200 pixels) on the path's
    LR-checked left map of one pair per workload, its four kernels replayed
    from a graph; minimum bytes = 2 B read + 2 B written per pixel (the
    label and size maps, 8 B per pixel more, stay in L2 at these sizes)."""
    import ctypes as C
    from paper_1802_07210_gb300 import _lib
    lib = _lib.lib()
    res = {}
    for key in ("vga_640", "kitti_1242"):
        wl, cfg = WORKLOADS[key]
        h, w = wl.spec.h, wl.spec.w
        L, R, _ = synth.workload_pair(wl, 400, cfg)
        pl = B.Pipeline(w, h, wl.params)
        dL = torch.empty((h, w), dtype=torch.int16, device=dev)
        pl.run(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev), dL)
        pl.close()
        out = torch.empty_like(dL)
        nb = lib.elas_speckle_workspace_bytes(w, h)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)

        def launch():
            rc = lib.elas_speckle(C.c_void_p(dL.data_ptr()), w, h, 1, 200, C.c_void_p(out.data_ptr()),
                                  C.c_void_p(ws.data_ptr()), nb, C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0
        us = _graph_us(torch, launch)
        gbs = 4.0 * w * h / (us * 1e-6) / 1e9
        removed = int(((out < 0) & (dL >= 0)).sum().item())
        res["%dx%d" % (w, h)] = {"us": us, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm_gbs,
                                 "pixels_removed": removed}
    return res


def census_timing(B, torch, dev, hbm_gbs):
    """The census variant at 640x480 D=256: the census kernel per record kind
    (both images per launch; minimum bytes = 2 image bytes read + 2 records
    written per pixel) and the whole one-pair pipeline per pair, next to the
    Sobel/SAD pipeline on the same pairs (L2 flushed before every pair)."""
    import ctypes as C
    from paper_1802_07210_gb300 import _lib
    lib = _lib.lib()
    wl, cfg = WORKLOADS["vga_640"]
    h, w = wl.spec.h, wl.spec.w
    L, R, _ = synth.workload_pair(wl, 300, cfg)
    tL, tR = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
    res = {}
    for W, nb in ((9, 32), (13, 32), (5, 16), (7, 16)):
        oL = torch.empty((h, w, nb), dtype=torch.uint8, device=dev)
        oR = torch.empty_like(oL)

        def launch():
            rc = lib.elas_census(C.c_void_p(tL.data_ptr()), C.c_void_p(tR.data_ptr()), w, h, w, W, nb,
                                 C.c_void_p(oL.data_ptr()), C.c_void_p(oR.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0
        us = _graph_us(torch, launch)
        gbs = 2.0 * w * h * (1 + nb) / (us * 1e-6) / 1e9
        res["census_%dx%d_%dB_us" % (W, W, nb)] = {"us": us, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm_gbs}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for key, ov in (("sobel_sad", {}), ("census_9x9_5x5", dict(census_support_w=9, census_dense_w=5)),
                    ("census_13x13_7x7", dict(census_support_w=13, census_dense_w=7))):
        pl = B.Pipeline(w, h, dict(wl.params, **ov))
        dL = torch.empty((h, w), dtype=torch.int16, device=dev)
        dR = torch.empty_like(dL)
        post = torch.empty((h, w), dtype=torch.float32, device=dev)
        ts = []
        for i in range(13):
            flush.fill_(i & 255)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record()
            pl.run(tL, tR, dL, dR, post)
            b_.record()
            b_.synchronize()
            if i >= 3:
                ts.append(a_.elapsed_time(b_))
        pl.close()
        res["pipeline_ms_per_pair_" + key] = float(np.median(ts))
    return res


def run_only(args, B, torch, dev):
    """One section alone (profiling runs)."""
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    class _Flush:
        def fill_(self, v):
            flush_buf.fill_(v)

    stream = torch.cuda.current_stream()
    steps = max(3, min(args.steps, 10))
    if args.only == "batch":
        peak = alu_peak(B, torch, dev, stream)[KERNEL_SAD_VARIANT] / 1e9
        return run_batch_section(B, torch, dev, stream, _Flush(), steps, args.batch_pairs, args.batch_distinct, peak,
                                 _peaks(), tune=not args.no_tune)
    if args.only == "mixed":
        return run_mixed_section(B, torch, dev, stream, _Flush(), steps, args.mixed_pairs, tune=not args.no_tune)
    if args.only == "accuracy":
        return run_accuracy_section(B, torch, dev)
    return {"offered": run_serve_section(B, torch, args.serve_seconds),
            "saturated": run_serve_section(B, torch, args.saturate_seconds, rate_per_camera=500.0, seed=6)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vga_640", choices=sorted(WORKLOADS))
    ap.add_argument("--pool", type=int, default=4, help="distinct pairs cycled through")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=64)
    ap.add_argument("--batch-distinct", type=int, default=64)
    ap.add_argument("--mixed-pairs", type=int, default=128)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--saturate-seconds", type=float, default=3.0,
                    help="length of the saturated serving schedule (offered load above the plain path's rate)")
    ap.add_argument("--skip-extra", action="store_true", help="only the plain-path line")
    ap.add_argument("--only", default=None, choices=["batch", "mixed", "serve", "accuracy"],
                    help="run only this section (its JSON object is printed alone)")
    ap.add_argument("--no-tune", action="store_true", help="batched sections keep the default tile shapes")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    wl, cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl, cfg)

    import torch
    import torch.distributed as dist
    from paper_1802_07210_gb300 import binding as B

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only:
        if rank == 0:
            print(json.dumps({args.only: run_only(args, B, torch, dev)}), flush=True)
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    w, h = wl.spec.w, wl.spec.h
    px = w * h
    pool = [synth.workload_pair(wl, replica_seed(rank, i), cfg) for i in range(args.pool)]
    imgs = [(torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)) for L, R, _ in pool]
    pl = B.Pipeline(w, h, wl.params)
    dL = torch.empty((h, w), dtype=torch.int16, device=dev)
    dR = torch.empty_like(dL)
    post = torch.empty((h, w), dtype=torch.float32, device=dev) if wl.postprocess else None
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    clean_buf = torch.zeros(256 << 20, dtype=torch.uint8, device=dev)

    class _Flush:
        """Writes 256 MB (evicting everything), then reads another 256 MB so
        that the dirty lines are written back before the timed region."""

        def fill_(self, v):
            flush_buf.fill_(v)
            clean_buf.max()

    flush = _Flush()
    stream = torch.cuda.current_stream()

    def step(i):
        L, R = imgs[i % len(imgs)]
        pl.run(L, R, dL, dR, post)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # ---- device-resident throughput of the plain path -------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    # the same steps again with the library's stage marks on (the marks cost
    # a few percent, so they are kept out of the headline steps)
    pl.set_profiling(True)
    for i in range(2):
        step(i)
    stage_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        step(i)
        stage_ms.append(pl.stats()["stage_ms"])  # events recorded by the library on this stream
    pl.set_profiling(False)
    total_ms = max_over_ranks(torch, dist, ws, sum(a.elapsed_time(b) for a, b in ev), dev)
    ms_step = total_ms / args.steps
    value = replica_throughput(ws, args.steps, px, total_ms) / 1e6
    st = pl.stats()
    stages = {k: float(np.mean([s[k] for s in stage_ms])) for k in STAGES}

    # ---- end to end through the host-buffer call -----------------------
    hL = [torch.from_numpy(L).pin_memory() for L, _, _ in pool]
    hR = [torch.from_numpy(R).pin_memory() for _, R, _ in pool]
    oL = torch.empty((h, w), dtype=torch.int16).pin_memory()
    opost = torch.empty((h, w), dtype=torch.float32).pin_memory() if wl.postprocess else None
    for i in range(3):
        pl.run_host(hL[i % len(hL)], hR[i % len(hR)], oL, None, opost)
    e2e_ms = 0.0
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl.run_host(hL[i % len(hL)], hR[i % len(hR)], oL, None, opost)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(torch, dist, ws, e2e_ms, dev)
    e2e = {"value": replica_throughput(ws, args.steps, px, e2e_ms) / 1e6, "unit": "Mpix/s",
           "h2d_bytes_per_step": 2 * px, "d2h_bytes_per_step": 2 * px + (4 * px if wl.postprocess else 0),
           "ms_per_step": e2e_ms / args.steps, "call": "elas_pipeline_run_host (pinned host buffers)"}

    # ---- roofline of the dense argmin kernel -----------------------------
    hbm_gbs, peak_kind = _peaks()
    probe = alu_peak(B, torch, dev, stream)
    peak = probe[KERNEL_SAD_VARIANT] / 1e9
    evals_pool = [pair_dense_evals(B, torch, wl, L, R, dev) for L, R, _ in pool]
    evals = float(np.mean([evals_pool[i % len(pool)] for i in range(args.steps)]))
    t_dense = stages["dense_argmin"]
    dense_bytes = DENSE_MIN_BYTES_PER_PX * px
    roof = {"kernel": "cell_kernel (dense argmin, both reference images in one launch)"}
    roof.update(dense_roofline(evals, dense_bytes, t_dense, peak, hbm_gbs, peak_kind))
    roof.update({
        "traffic": DENSE_TRAFFIC_BYTES.get(wl.name), "traffic_source": DENSE_TRAFFIC_SOURCE,
        "time": "mean of CUDA events around the launch, recorded by the library in a second pass of the timed "
                "steps (same pairs, same L2 flush)",
        "alu_peak_source": "measured: probe kernel running the dense matcher's SAD16 sequence (variant %d, the "
                           "fastest of the three) on registers over all SMs" % KERNEL_SAD_VARIANT,
        "probe_variants_gsad16": {str(k): v / 1e9 for k, v in probe.items()}})

    extra = {}
    if rank == 0 and not args.skip_extra:
        # each section reports on its own: an error in one is recorded in its
        # object and leaves the headline and the other sections standing
        sections = (
            ("accuracy", lambda: run_accuracy_section(B, torch, dev)),
            ("batch", lambda: run_batch_section(B, torch, dev, stream, flush, max(5, min(args.steps, 10)),
                                                args.batch_pairs, args.batch_distinct, peak, (hbm_gbs, peak_kind),
                                                tune=not args.no_tune)),
            ("batch_census", lambda: run_batch_section(B, torch, dev, stream, flush, max(5, min(args.steps, 10)),
                                                       args.batch_pairs, args.batch_distinct, peak,
                                                       (hbm_gbs, peak_kind), tune=not args.no_tune,
                                                       overrides=dict(census_support_w=9, census_dense_w=5))),
            ("mixed_batch", lambda: run_mixed_section(B, torch, dev, stream, flush, max(5, min(args.steps, 10)),
                                                      args.mixed_pairs, tune=not args.no_tune)),
            ("serving", lambda: run_serve_section(B, torch, args.serve_seconds)),
            ("serving_saturated", lambda: run_serve_section(B, torch, args.saturate_seconds, rate_per_camera=500.0,
                                                            seed=6)),
        )
        for key, fn in sections:
            try:
                extra[key] = fn()
            except Exception as e:  # noqa: BLE001
                extra[key] = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": wl.name, "w": w, "h": h, "disp_max": wl.disp_max,
                           "pairs_per_step": 1, "pool": args.pool, "path": "plain one-pair path (elas_pipeline_run)",
                           "triangulation": "GPU",
                           "l2": "flushed before every timed step (256 MB write, then 256 MB read so no dirty lines remain)"},
                "pairs_per_s": replica_throughput(ws, args.steps, 1, total_ms),
                "support_points": st["n_support"], "triangles": [st["n_tri_left"], st["n_tri_right"]],
                "stages_ms": stages, "clocks": clk, "e2e": e2e,
                "gpu_launches": KERNELS_PER_STEP[bool(wl.postprocess)] * args.steps, "roofline": roof}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, cfg)
        # the long accuracy object first; the throughput sections and a
        # compact summary close the line
        line.update(extra)
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def summary(line):
    """The figures of every section in one small object."""
    out = {"plain_mpix_per_s": line["value"], "plain_pairs_per_s": line["pairs_per_s"],
           "e2e_mpix_per_s": line["e2e"]["value"],
           "dense": {"bound": line["roofline"]["bound"], "frac": line["roofline"]["frac"],
                     "frac_alu": line["roofline"]["alu"]["frac"], "frac_hbm": line["roofline"]["hbm"]["frac"],
                     "launch_us": line["roofline"]["launch_us"]}}
    b = line.get("batch", {})
    if "pairs_per_s" in b:
        out["batch_64x1242x375"] = {"pairs_per_s": b["pairs_per_s"], "plain_pairs_per_s": b["plain_pairs_per_s"],
                                    "speedup": b["speedup_vs_plain"], "distinct_pairs": b["distinct_pairs"],
                                    "dense_bound": b["roofline_dense"]["bound"],
                                    "dense_frac": b["roofline_dense"]["frac"],
                                    "dense_frac_alu": b["roofline_dense"]["alu"]["frac"]}
    bc = line.get("batch_census", {})
    if "pairs_per_s" in bc:
        out["batch_census_9x9_5x5"] = {"pairs_per_s": bc["pairs_per_s"], "plain_pairs_per_s": bc["plain_pairs_per_s"],
                                       "speedup": bc["speedup_vs_plain"]}
    m = line.get("mixed_batch", {})
    if "pairs_per_s" in m:
        out["mixed_128"] = {"pairs_per_s": m["pairs_per_s"], "plain_pairs_per_s": m["plain_pairs_per_s"],
                            "speedup": m["speedup_vs_plain"]}
    for key in ("serving", "serving_saturated"):
        sv = line.get(key, {})
        if "continuous_batching" in sv:
            cb, pp = sv["continuous_batching"], sv["plain_per_pair"]
            out[key] = {"offered_pairs_per_s": sv["offered_pairs_per_s"], "seconds": sv["seconds"],
                        "batched": {k: cb[k] for k in ("pairs_per_s", "p50_ms", "p99_ms")},
                        "plain": {k: pp[k] for k in ("pairs_per_s", "p50_ms", "p99_ms")}}
    return out


def dense_work(work, prm, w, h):
    """Candidate evaluations of the dense step, both reference images:
    |S(p)| = |(grid(cell) U plane window) within the admissible range| per
    matched pixel (each a 16-byte SAD)."""
    G = prm.grid_size
    sr = prm.sradius
    total = 0
    vv, uu = np.mgrid[0:h, 0:w]
    for side in (0, 1):
        ref = work["descR"] if side else work["descL"]
        dp = (work["dpR"] if side else work["dpL"]).astype(np.int64)
        grid = (work["gridR"] if side else work["gridL"]).view(np.uint32)
        tex = np.abs(ref.astype(np.int32) - 128).sum(-1)
        ok = (uu >= 2) & (uu <= w - 3) & (vv >= 2) & (vv <= h - 3) & (tex >= prm.match_texture) & (dp >= 0)
        dlim = np.minimum(prm.disp_max, (w - 3 - uu) if side else (uu - 2))
        gh, gw = grid.shape[:2]
        for cy in range(gh):
            for cx in range(gw):
                bits = np.unpackbits(grid[cy, cx].view(np.uint8), bitorder="little")
                cand = np.nonzero(bits)[0]
                cand = cand[(cand >= prm.disp_min) & (cand <= prm.disp_max)]
                ys, xs = slice(cy * G, min(h, cy * G + G)), slice(cx * G, min(w, cx * G + G))
                m = ok[ys, xs]
                if not m.any():
                    continue
                dl = dlim[ys, xs][m]
                d0 = dp[ys, xs][m]
                cnt = np.searchsorted(cand, dl, side="right")
                inmask = np.zeros(prm.disp_max + 2, bool)
                inmask[cand] = True
                for k in range(-sr, sr + 1):
                    d = d0 + k
                    valid = (d >= prm.disp_min) & (d <= dl)
                    cnt = cnt + (valid & ~inmask[np.clip(d, 0, prm.disp_max + 1)])
                total += int(cnt.sum())
    return total


# DRAM bytes (read + write) of one cell_kernel launch, from one ncu capture of
# the kernel as it is now (dram__bytes_read.sum + dram__bytes_write.sum);
# to be taken again whenever the kernel changes, and reported as null until
# then.  The last capture (11,162,112 bytes at 640x480 D=256) predates the
# list walk's predicate, so the entry is empty.
DENSE_TRAFFIC_BYTES = {}
DENSE_TRAFFIC_SOURCE = ("null: the kernel changed after its last capture (ncu --metrics dram__bytes_read.sum,"
                        "dram__bytes_write.sum,gpu__time_duration.sum --clock-control none -k regex:cell_kernel -s 2 "
                        "-c 1 on python bench.py --steps 3 --warmup 3 --no-cpu-baseline --skip-extra: 11,162,112 bytes "
                        "for the previous build, reads only, below the minimum bytes because the descriptors written "
                        "just before stay partly in L2)")

KERNEL_SAD_VARIANT = 2  # the probe variant whose instruction sequence the dense matcher uses


def dense_roofline(evals, min_bytes, t_ms, peak_gsad, hbm_gbs, peak_kind):
    """Both roofs of a dense launch (algorithmic work over its measured time)
    and the binding one: the roof whose own lower bound on the time is the
    larger (HBM at these candidate counts: about 10 SAD16 per pixel and
    image against 40 bytes per pixel)."""
    t = t_ms * 1e-3
    alu = {"achieved": evals / t / 1e9, "peak": peak_gsad, "unit": "G SAD16/s",
           "frac": evals / t / 1e9 / peak_gsad, "algorithmic_evals": evals,
           "lower_bound_us": evals / (peak_gsad * 1e9) * 1e6}
    hbm = {"achieved": min_bytes / t / 1e9, "peak": hbm_gbs, "unit": "GB/s",
           "frac": min_bytes / t / 1e9 / hbm_gbs, "algorithmic_bytes": min_bytes,
           "lower_bound_us": min_bytes / (hbm_gbs * 1e9) * 1e6,
           "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % peak_kind}
    bound = "hbm" if hbm["lower_bound_us"] >= alu["lower_bound_us"] else "alu"
    top = hbm if bound == "hbm" else alu
    return {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "launch_us": t_ms * 1e3, "alu": alu, "hbm": hbm}


def alu_peak(B, torch, dev, stream):
    """SAD16/s of the probe kernel (the SAD sequence alone, registers only,
    every SM): the ALU ceiling of the matchers."""
    import ctypes as C
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sm * 8, 256, 2048
    scratch = torch.empty(blocks * threads, dtype=torch.int32, device=dev)
    res = {}
    for variant in (0, 1, 2):
        args = (variant, blocks, threads, iters, C.c_void_p(scratch.data_ptr()), C.c_void_p(stream.cuda_stream))
        B.check(B.lib().elas_probe_sad16(*args))
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            B.check(B.lib().elas_probe_sad16(*args))
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        res[variant] = blocks * threads * iters * 8 / (min(ts) * 1e-3)
    return res


if __name__ == "__main__":
    main()
