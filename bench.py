"""Throughput of the ELAS path on GB300: Mpix/s and pairs/s at 640x480 with
256 disparities (one stereo pair per step, the whole path: descriptors,
support points, host triangulation, plane prior, dense matching, LR check,
post-processing).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas, one per
GPU (pairs are independent; there is no collective on the data path).
``--impl reference`` times the CPU oracle on the host cores instead.
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
KERNELS_PER_STEP = 11  # descriptor 1, support 4, prior binning 1, dense 1, LR 1, post 4


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


def cpu_baseline(wl, cfg, seconds=12.0):
    """The oracle as it stands, single-threaded, on whole pairs of the
    workload until about `seconds` of CPU work (at least one pair)."""
    import oracle
    oracle.lib()
    n, t = 0, 0.0
    while t < seconds or n == 0:
        L, R, _ = synth.workload_pair(wl, 100 + n, cfg)
        t0 = time.perf_counter()
        oracle.pipeline(L, R, wl.params, postprocess_on=wl.postprocess)
        t += time.perf_counter() - t0
        n += 1
        if n >= 8:
            break
    px = wl.spec.w * wl.spec.h
    return {"value": n * px / t / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": "%d whole %dx%d pairs through the oracle pipeline (%.1f s)" % (n, wl.spec.w, wl.spec.h, t),
            "pairs_per_s": n / t}


def run_reference(args, wl, cfg):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.lib()
    px = wl.spec.w * wl.spec.h
    pairs = [synth.workload_pair(wl, i, cfg) for i in range(min(4, args.steps + args.warmup))]
    for i in range(args.warmup):
        L, R, _ = pairs[i % len(pairs)]
        oracle.pipeline(L, R, wl.params, postprocess_on=wl.postprocess)
    t = 0.0
    for i in range(args.steps):
        L, R, _ = pairs[i % len(pairs)]
        t0 = time.perf_counter()
        oracle.pipeline(L, R, wl.params, postprocess_on=wl.postprocess)
        t += time.perf_counter() - t0
    val = args.steps * px / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": wl.name, "w": wl.spec.w, "h": wl.spec.h,
                                            "disp_max": wl.disp_max, "sample": "whole pairs"},
            "pairs_per_s": args.steps / t,
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                             "sample": "%d whole %s pairs, one per step" % (args.steps, wl.name)},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="vga_640", choices=sorted(WORKLOADS))
    ap.add_argument("--pool", type=int, default=4, help="distinct pairs cycled through")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    w, h = wl.spec.w, wl.spec.h
    px = w * h
    pool = [synth.workload_pair(wl, rank * 1000 + i, cfg) for i in range(args.pool)]
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

    # ---- device-resident throughput ------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    tri_ms = []
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
        tri_ms.append(pl.stats()["triangulate_ms"])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_all = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_all, op=dist.ReduceOp.MAX)
    total_ms = float(t_all.item())
    ms_step = total_ms / args.steps
    value = ws * args.steps * px / (total_ms / 1e3) / 1e6
    st = pl.stats()

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
    t_e = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
    e2e_ms = float(t_e.item())
    e2e = {"value": ws * args.steps * px / (e2e_ms / 1e3) / 1e6, "unit": "Mpix/s",
           "h2d_bytes_per_step": 2 * px, "d2h_bytes_per_step": 2 * px + (4 * px if wl.postprocess else 0),
           "ms_per_step": e2e_ms / args.steps}

    # ---- per-stage kernel times (C-ABI calls bracketed by events) -------
    stages, work = stage_times(B, torch, wl, pool[0], dev, stream, flush, reps=max(5, min(args.steps, 20)))
    hbm_gbs, peak_kind = _peaks()
    prm = B.as_params(wl.params)
    evals = dense_work(work, prm, w, h)
    probe = alu_peak(B, torch, dev, stream)
    t_dense = stages["dense_match_ms"]
    achieved = evals / (t_dense * 1e-3) / 1e9
    peak = probe[0] / 1e9
    # algorithmic HBM bytes of the same launch: both descriptor images read
    # once (32 B/px), grid vectors and meshes (small), two int16 maps written
    dense_bytes = 2 * (16 + 16 + 2) * px
    roof = {"kernel": "cell_kernel<kDenseFused> (prior + dense argmin, both reference images)",
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "G SAD16/s", "frac": achieved / peak,
            "traffic": None, "algorithmic_evals": evals,
            "peak_source": "measured: probe kernel running the same SAD16 sequence on registers over all SMs",
            "probe_variants_gsad16": {str(k): v / 1e9 for k, v in probe.items()},
            "hbm": {"achieved_gbs": dense_bytes / (t_dense * 1e-3) / 1e9, "peak_gbs": hbm_gbs,
                    "frac": dense_bytes / (t_dense * 1e-3) / 1e9 / hbm_gbs,
                    "peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % peak_kind}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": wl.name, "w": w, "h": h, "disp_max": wl.disp_max,
                           "pairs_per_step": 1, "pool": args.pool, "path": "plain one-pair path",
                           "l2": "flushed before every timed step (256 MB write, then 256 MB read so no dirty lines remain)"},
                "pairs_per_s": ws * args.steps / (total_ms / 1e3),
                "triangulate_ms_median": float(np.median(tri_ms)),
                "support_points": st["n_support"], "triangles": [st["n_tri_left"], st["n_tri_right"]],
                "stages_ms": stages, "clocks": clk, "e2e": e2e,
                "gpu_launches": KERNELS_PER_STEP * args.steps, "roofline": roof}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, cfg)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def stage_times(B, torch, wl, pair, dev, stream, flush, reps=10):
    """Median device time of each stage's C-ABI call on one pair, plus the
    inputs needed to count the dense matcher's algorithmic work."""
    L, R, _ = pair
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
    dl, dr = B.elas_dense_match(descL, descR, prm, lst, n, triL, triR, sp["grid_L"], sp["grid_R"])
    dl2, dr2 = dl.clone(), dr.clone()
    calls = {
        "descriptors_ms": lambda: B.elas_descriptors(tL, tR),
        "support_ms": lambda: B.elas_support_points(descL, descR, prm),
        "dense_match_ms": lambda: B.elas_dense_match(descL, descR, prm, lst, n, triL, triR, sp["grid_L"],
                                                     sp["grid_R"]),
        "plane_prior_L_ms": lambda: B.elas_plane_prior(lst, triL, w, h, prm, False),
        "dense_argmin_L_ms": lambda: B.elas_dense_argmin(descL, descR, prm, dpL, sp["grid_L"], False),
        "lr_check_ms": lambda: B.elas_lr_check(dl2, dr2, prm.lr_threshold, masks=False),
        "postprocess_ms": lambda: B.elas_postprocess(dl, prm),
    }
    out = {}
    for name, fn in calls.items():
        fn()
        ts = []
        for i in range(reps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.median(ts))
    work = dict(descL=descL.cpu().numpy(), descR=descR.cpu().numpy(), dpL=dpL.cpu().numpy(),
                dpR=dpR.cpu().numpy(), gridL=sp["grid_L"].cpu().numpy(), gridR=sp["grid_R"].cpu().numpy())
    return out, work


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
