"""Benchmark of the Binary Stereo Matching hot path on GB300.

One step = the whole path on one stereo pair with inputs already resident in HBM: describe (left and
right view), the fused cost + aggregation + WTA kernel (both reference views) and the left/right
check + refinement. Metric: Gpix*disp/s = width * height * dmax per pair / step time.

Default run (no flags): the 3840 x 2160 RGB8 pair with dmax 256 (n = 256 bits, S = 31, aggregation
window 5, k = n/4, R = 15) is the headline line; the same JSON line carries
  "batched": the batch of 64 uneven pairs in persistent launches against the per-pair calls, both
             timed in this process on this build, with the launch-gap bound of the per-pair path;
  "served":  a 10,000-request Poisson stream (rho = 0.7 of the engine's measured capacity) through the
             continuous-batching engine against one-at-a-time processing of the same trace.

  python bench.py [--gpus N --steps K --warmup W] [--config c1|c2|c3|c4|c5] [--impl ours|reference]

An explicit --config runs that configuration alone. Multi-GPU (torchrun, one process per GPU) runs
independent replicas: every rank processes its own pair, nothing is exchanged, value = all ranks'
pixels*disparities / max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {
    "c1": dict(w=450, h=375, dmax=60, radiometric=False, seed=1,
               name="450x375 RGB8 pair (Teddy-shaped), dmax 60"),
    "c2": dict(w=1390, h=1110, dmax=256, radiometric=True, seed=2,
               name="1390x1110 RGB8 pair, dmax 256, radiometric right view"),
    "c4": dict(w=3840, h=2160, dmax=256, radiometric=False, seed=4,
               name="3840x2160 RGB8 pair, dmax 256"),
    "c3": dict(count=64, seed=3, name="batch of 64 uneven pairs: w U[320,1920], h U[240,1080], dmax {64,128,192,256}"),
    "c5": dict(seed=5, name="serving stream: Poisson arrivals, sizes {640x480,1280x720,1920x1080,3840x2160} x dmax "
                            "{64,128,256}, continuous batching vs one-at-a-time"),
}
N_BITS, WINDOW_S, AGG, VOTE_R = 256, 31, 5, 15
PAIR_SEED = 11
METRIC = "Gpix*disp/s"
L2_FLUSH_BYTES = 256 << 20
SMS, MAX_SM_MHZ = 152, 2070  # the GB300's SM count and maximum SM clock
ISSUE_PER_CLK_SM = 4 * 32    # four schedulers per SM, one warp instruction (32 lanes) each per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default="", choices=[""] + sorted(CONFIGS),
                    help="run one configuration alone (default: c4 with the batched c3 and served c5 objects)")
    ap.add_argument("--no-batched", action="store_true", help="default run without the batched (c3) object")
    ap.add_argument("--no-served", action="store_true", help="default run without the served (c5) object")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cost-rows", type=int, default=0, help="rows per CTA of the cost kernel (0: heuristic)")
    ap.add_argument("--cost-popc-plain", type=int, default=0, help="1: plain popcount in the cost kernel")
    ap.add_argument("--batch-rows", type=int, default=0, help="rows per task of the batched cost kernel (0: 64)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--cost-variant", type=int, default=0,
                    help="cost kernel: 1 one column per lane, 2 two columns, 3 tensor cores (0: autotuned)")
    ap.add_argument("--describe-variant", type=int, default=0,
                    help="describe kernel: 0 auto, 1 thread per pixel, 2 warp per pixel")
    ap.add_argument("--describe-copies", type=int, default=0,
                    help="tile copies of the warp-per-pixel describe kernel (0: one; 1..4)")
    ap.add_argument("--n-bits", type=int, default=N_BITS, help="descriptor length n (32 ... 4096)")
    ap.add_argument("--sgm", default="", help="P1,P2,paths: semi-global aggregation of both cost volumes")
    ap.add_argument("--quality", action="store_true",
                    help="bad-pixel rates against the generator's ground truth: mask ablation, radiometric 3x3")
    ap.add_argument("--sweep-n", action="store_true",
                    help="speed for every descriptor length 32 ... 4096 on the chosen pair config (Fig. 3b)")
    ap.add_argument("--requests", type=int, default=10000, help="serving stream length (c5)")
    ap.add_argument("--rho", type=float, default=0.7, help="arrival rate as a fraction of measured capacity (c5)")
    ap.add_argument("--lanes", type=int, default=2, help="serving lanes (c5)")
    ap.add_argument("--max-batch", type=int, default=16, help="serving batch limit (c5)")
    ap.add_argument("--batch-work", type=float, default=1.0,
                    help="serving cap on a batch's pixels x disparities, in units of one 3840x2160x256 pair (c5)")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, max clock, throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_traffic(kernel_file, workload_key):
    """ncu DRAM traffic per launch recorded in profiles/, valid only for the unchanged kernel source."""
    src = os.path.join(ROOT, "paper_1402_2020_gb300", "csrc", kernel_file)
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, fn)):
            m = re.match(r"traffic_per_launch:\s*(\w+)\s+(\S+)\s+bytes=(\d+)\s+source_sha256=(\w+)", line.strip())
            if m and m.group(1) == workload_key and m.group(2) == kernel_file and m.group(4) == digest:
                return int(m.group(3))
    return None


_SAMPLE_CACHE = {}


def oracle_sample(cfg, rows):
    """The oracle as it stands on a band of `rows` rows of the workload: returns (seconds, pix*disp)."""
    from oracle import oracle
    from paper_1402_2020_gb300 import synth

    if "count" in cfg:  # batch workload: sample the first pair of the batch
        w, h, dmax, seed = synth.batch_shapes(cfg["count"], seed=cfg["seed"])[0]
        cfg = dict(w=w, h=h, dmax=dmax, seed=seed, radiometric=False)
    elif "w" not in cfg:  # request stream: sample its 1280x720, dmax 128 class
        cfg = dict(w=1280, h=720, dmax=128, seed=cfg["seed"], radiometric=False)
    key = (cfg["w"], cfg["h"], cfg["dmax"], cfg["seed"], cfg["radiometric"])
    if key not in _SAMPLE_CACHE:
        _SAMPLE_CACHE[key] = synth.stereo_pair(*key)
    left, right, _ = _SAMPLE_CACHE[key]
    pairs = synth.pair_table(N_BITS, WINDOW_S, seed=PAIR_SEED)
    y0 = cfg["h"] // 2 - rows // 2
    l = np.ascontiguousarray(left[y0:y0 + rows])
    r = np.ascontiguousarray(right[y0:y0 + rows])
    t = time.perf_counter()
    oracle.pipeline(l, r, pairs, cfg["dmax"], win=AGG, R=VOTE_R)
    dt = time.perf_counter() - t
    return dt, cfg["w"] * rows * cfg["dmax"]


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank floats over all ranks (identity on one rank). Replicas share no
    data, so this reduction of their timings is the only collective the benchmark makes."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def run_reference(args, cfg, world, rank):
    """The oracle as it stands, single-threaded on one pinned host core, on a bounded row band of the
    workload per step (the band keeps the whole --steps K --warmup W run within a few minutes)."""
    if rank != 0:
        return
    rows = 8 if cfg.get("w", 0) >= 3000 else 16
    if "count" in cfg:
        from paper_1402_2020_gb300 import synth

        w0 = synth.batch_shapes(cfg["count"], seed=cfg["seed"])[0][0]
        cfg = dict(cfg, w=w0)
    elif "w" not in cfg:
        cfg = dict(cfg, w=1280)

    def run():
        times = []
        for i in range(args.warmup + args.steps):
            dt, units = oracle_sample(cfg, rows)
            if i >= args.warmup:
                times.append(dt)
        return times, units

    (times, units), core = pinned_to_one_core(run)
    t = float(np.mean(times))
    v = units / t / 1e9
    nproc, model = host_cpu()
    sample = f"{cfg['w']}x{rows} row band of the workload per step, whole oracle pipeline, single thread pinned to " \
             f"host core {core}"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": cfg["name"], "n_bits": N_BITS, "agg_window": AGG, "sample": sample},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                             "nproc": nproc, "cpu_model": model},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, cfg, world, rank, local):
    """Config 3: one bsm_batch_run per step (persistent launches from a CUDA graph) against the same 64 pairs
    through the per-pair calls (four C-ABI calls per pair), both timed here on this build. The per-pair
    path is timed twice: as issued (`plain`) and with the whole step enqueued behind a GPU-side delay so
    that its kernels run back to back (`plain_gap_free`): the ratio bounds what removing launch gaps alone
    can give. Returns the JSON object."""
    import torch

    from paper_1402_2020_gb300 import bsm, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shapes = synth.batch_shapes(cfg["count"], seed=cfg["seed"] + 1000 * rank)
    pairs = synth.pair_table(N_BITS, WINDOW_S, seed=PAIR_SEED)
    params = bsm.make_params(pairs, window_S=WINDOW_S, agg_window=AGG, dmax=256, vote_radius=VOTE_R)
    ctx = bsm.bsm_create(params)
    bsm.bsm_set_tuning(ctx, args.cost_rows, args.cost_popc_plain, args.batch_rows, 0, args.describe_variant,
                       args.describe_copies)
    nw = N_BITS // 32
    ts = []
    for (w, h, dmax, seed) in shapes:
        l, r, _ = synth.stereo_pair(w, h, dmax, seed)
        t = {"w": w, "h": h, "dmax": dmax, "rgbL": torch.from_numpy(l).to(dev), "rgbR": torch.from_numpy(r).to(dev)}
        for k in ("BL", "PhiL", "BR", "PhiR"):
            t[k] = torch.empty((h, w, nw), dtype=torch.int32, device=dev)
        for k in ("dispL", "dispR", "out"):
            t[k] = torch.empty((h, w), dtype=torch.int32, device=dev)
        ts.append(t)
    descs = [bsm.pair_desc(t["rgbL"], t["rgbR"], t["w"], t["h"], 3 * t["w"], t["dmax"], t["BL"], t["PhiL"], t["BR"],
                           t["PhiR"], t["dispL"], t["dispR"], t["out"]) for t in ts]
    units = sum(t["w"] * t["h"] * t["dmax"] for t in ts)
    stream = torch.cuda.Stream(device=dev)
    s = stream.cuda_stream
    bsm.bsm_reserve(ctx, max(t["w"] for t in ts), max(t["h"] for t in ts))
    bsm.bsm_reserve_batch(ctx, sum(t["w"] * t["h"] for t in ts))
    if not args.no_autotune and args.batch_rows == 0:
        from paper_1402_2020_gb300 import autotune

        with torch.cuda.stream(stream):
            autotune.tune_batch(ctx, descs, N_BITS, AGG)

    def batched():
        bsm.bsm_batch_run(ctx, descs, s)

    def plain():
        for t in ts:
            w, h, dmax = t["w"], t["h"], t["dmax"]
            bsm.bsm_describe(ctx, t["rgbL"], w, h, 3 * w, t["BL"], t["PhiL"], s)
            bsm.bsm_describe(ctx, t["rgbR"], w, h, 3 * w, t["BR"], t["PhiR"], s)
            bsm.bsm_cost_aggregate_wta(ctx, t["BL"], t["PhiL"], t["BR"], t["PhiR"], w, h, dmax, t["dispL"],
                                       t["dispR"], None, s)
            bsm.bsm_refine(ctx, t["rgbL"], 3 * w, t["dispL"], t["dispR"], w, h, dmax, t["out"], s)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                fn()
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            for i in range(args.steps):
                e0[i].record(stream)
                fn()
                e1[i].record(stream)
            torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in zip(e0, e1)]))

    def gap_free(fn, reps=3):
        # the GPU spins for a bounded time (torch's clock-based sleep kernel) while the host enqueues the
        # whole step behind it; the step's kernels then run back to back without launch gaps
        out = []
        with torch.cuda.stream(stream):
            for _ in range(reps):
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda._sleep(int(0.2 * MAX_SM_MHZ * 1e6))
                t0 = time.perf_counter()
                a.record(stream)
                fn()
                b.record(stream)
                host_s = time.perf_counter() - t0
                torch.cuda.synchronize()
                out.append((a.elapsed_time(b), host_s))
        return float(np.mean([o[0] for o in out])), max(o[1] for o in out)

    clk = Clocks(local)
    clk.start()
    t_batch = timed(batched)
    clocks = clk.stop()
    t_plain = timed(plain)
    t_free, host_enqueue_s = gap_free(plain)
    assert bsm.bsm_last_error(ctx) == bsm.BSM_OK
    t_batch, t_plain, t_free = max_over_ranks([t_batch, t_plain, t_free], world, dev)
    value = world * units / (t_batch * 1e-3) / 1e9
    tuning = bsm.bsm_get_tuning(ctx)
    # the batch: four persistent launches, plus one tensor-core cost launch per pair of at least
    # 1280 x 720 x 128 pixel-disparities; the per-pair calls: colour pre-pass and describe per view, the
    # cost stage's kernels, the refinement-word pass, the block ordering and refine
    n_tc = sum(1 for t in ts if t["w"] * t["h"] * t["dmax"] >= 1280 * 720 * 128) if tuning["cost_variant"] in (0, 3) else 0
    plain_launches = sum(4 + bsm.bsm_cost_plan(ctx, t["w"], t["h"], t["dmax"])["launches"] + 3 for t in ts)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg["name"], "n_bits": N_BITS, "agg_window": AGG, "pairs": len(ts),
                   "pixels": sum(t["w"] * t["h"] for t in ts), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (all 64 pairs' planes resident, about 7 GB)"},
        "pairs_per_s": world * len(ts) / (t_batch * 1e-3),
        "plain": {"value": world * units / (t_plain * 1e-3) / 1e9, "ms_per_step": t_plain,
                  "pairs_per_s": world * len(ts) / (t_plain * 1e-3), "launches_per_step": plain_launches},
        "batched_over_plain": t_plain / t_batch,
        "bound": {"plain_gap_free_ms": t_free, "plain_ms": t_plain,
                  "launch_gap_share_of_plain": 1.0 - t_free / t_plain,
                  "plain_over_gap_free": t_plain / t_free,
                  "host_enqueue_s": host_enqueue_s, "delay_s": 0.2,
                  "note": "plain_gap_free: the per-pair calls enqueued behind a 0.2 s GPU-side delay so their kernels "
                          "run back to back; valid while host_enqueue_s < delay_s"},
        "gpu_launches": (4 + n_tc) * args.steps,
        "clocks": clocks,
        "tuning": tuning,
    }
    bsm.bsm_destroy(ctx)
    return line


def run_serving(args, cfg, world, rank, local):
    """Config 5: a Poisson request stream through the continuous-batching engine, against the same trace
    processed one request at a time through the host-buffer C-ABI call. Returns the JSON object."""
    import torch

    from paper_1402_2020_gb300 import bsm, synth

    torch.cuda.set_device(local)
    pairs = synth.pair_table(N_BITS, WINDOW_S, seed=PAIR_SEED)
    params = bsm.make_params(pairs, window_S=WINDOW_S, agg_window=AGG, dmax=256, vote_radius=VOTE_R)
    classes = [(w, h, d) for (w, h) in synth.SERVE_SIZES for d in synth.SERVE_DMAX]
    data = {}
    for i, (w, h, d) in enumerate(classes):
        l, r, _ = synth.stereo_pair(w, h, d, cfg["seed"] * 100 + i + 1000 * rank)
        data[(w, h, d)] = (torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory(),
                           torch.empty((h, w), dtype=torch.int32).pin_memory())
    srv = bsm.bsm_server_create(params, lanes=args.lanes, max_batch=args.max_batch,
                                max_batch_work=int(args.batch_work * 3840 * 2160 * 256))
    ctx = bsm.bsm_create(params)
    rng = np.random.default_rng(cfg["seed"] + rank)

    def submit(i, c):
        l, r, o = data[c]
        st = bsm.bsm_server_submit(srv, i, l, r, c[0], c[1], 3 * c[0], c[2], o)
        assert st == bsm.BSM_OK, st

    # warm-up (graph capture, pools) and capacity: a flat-out burst
    for i in range(2 * len(classes)):
        submit(i, classes[i % len(classes)])
    bsm.bsm_server_drain(srv)
    while bsm.bsm_server_poll(srv, 256, 0):
        pass
    n_cap = 240
    burst = [classes[int(k)] for k in rng.integers(0, len(classes), size=n_cap)]
    t0 = time.perf_counter()
    for i, c in enumerate(burst):
        submit(10 ** 6 + i, c)
    bsm.bsm_server_drain(srv)
    capacity = n_cap / (time.perf_counter() - t0)
    while bsm.bsm_server_poll(srv, 256, 0):
        pass

    # capacity of one-at-a-time processing on the same burst
    t0 = time.perf_counter()
    for c in burst:
        l, r, o = data[c]
        bsm.bsm_match_host(ctx, l.data_ptr(), r.data_ptr(), c[0], c[1], 3 * c[0], c[2], o.data_ptr())
    capacity_plain = n_cap / (time.perf_counter() - t0)

    trace = synth.request_trace(args.requests, args.rho * capacity, seed=cfg["seed"] + rank)
    units = sum(w * h * d for (_, w, h, d) in trace)

    def served():
        done = {}
        start = time.perf_counter() + 0.05

        def producer():
            for i, (ta, w, h, d) in enumerate(trace):
                delay = start + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                submit(i, (w, h, d))

        th = threading.Thread(target=producer)
        th.start()
        while len(done) < len(trace):
            for cid, st, _ in bsm.bsm_server_poll(srv, 512, 2000):
                assert st == bsm.BSM_OK, st
                done[cid] = time.perf_counter()
        th.join()
        lat = np.array([done[i] - (start + trace[i][0]) for i in range(len(trace))])
        return lat, max(done.values()) - start

    def plain():
        done = []
        start = time.perf_counter() + 0.05
        for ta, w, h, d in trace:
            delay = start + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            l, r, o = data[(w, h, d)]
            bsm.bsm_match_host(ctx, l.data_ptr(), r.data_ptr(), w, h, 3 * w, d, o.data_ptr())
            done.append(time.perf_counter())
        lat = np.array([done[i] - (start + trace[i][0]) for i in range(len(trace))])
        return lat, done[-1] - start

    clk = Clocks(local)
    clk.start()
    lat_s, wall_s = served()
    clocks = clk.stop()
    stats = bsm.bsm_server_get_stats(srv)
    lat_p, wall_p = plain()
    bsm.bsm_server_destroy(srv)
    bsm.bsm_destroy(ctx)

    def summary(lat, wall):
        return {"pairs_per_s": len(trace) / wall, "gpix_disp_per_s": units / wall / 1e9,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3), "wall_s": wall}

    s_sum, p_sum = summary(lat_s, wall_s), summary(lat_p, wall_p)
    line = {
        "metric": METRIC, "value": s_sum["gpix_disp_per_s"] * world, "unit": METRIC, "n_gpus": world,
        "steps": len(trace), "warmup": 2 * len(classes), "ms_per_step": wall_s * 1e3 / len(trace),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg["name"], "requests": len(trace), "rho": args.rho, "lanes": args.lanes,
                   "max_batch": args.max_batch, "max_batch_work_4k_units": args.batch_work,
                   "arrival_rate_per_s": args.rho * capacity,
                   "n_bits": N_BITS, "agg_window": AGG, "parallelism": f"replicas x{world}"},
        "capacity_pairs_per_s": capacity, "capacity_one_at_a_time_pairs_per_s": capacity_plain,
        "capacity_ratio": capacity / capacity_plain,
        "served": s_sum, "one_at_a_time": p_sum,
        "p99_speedup": p_sum["p99_ms"] / s_sum["p99_ms"],
        "engine": stats, "clocks": clocks,
    }
    return line


def torch_dist_done():
    import torch.distributed as dist

    dist.destroy_process_group()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


_INT_RATES = None


def int_rates():
    """Issue rates (lanes per clock per SM) of POPC and the ALU-pipe instructions: the summary the
    issue-rate probe wrote under profiles/ while its source is unchanged, else a live run of the probe.
    Returns (rates, basis)."""
    global _INT_RATES
    if _INT_RATES is None:
        from paper_1402_2020_gb300 import peaks

        rec = peaks.load()
        if rec is not None:
            _INT_RATES = (rec, f"issue-rate probe, {os.path.relpath(peaks.SUMMARY, ROOT)} "
                               f"(probe source sha256 {peaks.source_hash()})")
        else:
            _INT_RATES = (peaks.measure(), "issue-rate probe run live (no summary for this probe source)")
    return _INT_RATES


def popc_peak():
    """Masked 32-bit popcounts per second: SMs x POPC lanes per clock x the maximum SM clock (Gpopc/s)."""
    from paper_1402_2020_gb300 import peaks

    rates, basis = int_rates()
    r = peaks.rounded(rates, "POPC")
    return SMS * r * MAX_SM_MHZ * 1e6 / 1e9, f"{SMS} SMs x {r:.0f} POPC/clk x {MAX_SM_MHZ} MHz ({basis})"


def alu_peak():
    """32-bit integer lane operations per second on the ALU pipe (LOP3 / IMNMX / VABSDIFF4 rate) (Gop/s)."""
    from paper_1402_2020_gb300 import peaks

    rates, basis = int_rates()
    r = peaks.rounded(rates, "LOP3")
    return SMS * r * MAX_SM_MHZ * 1e6 / 1e9, f"{SMS} SMs x {r:.0f} ALU lanes/clk (LOP3) x {MAX_SM_MHZ} MHz ({basis})"


def host_cpu():
    """(cores the machine has, CPU model name) of the host the oracle is timed on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def pinned_to_one_core(fn):
    """Runs fn() with this process pinned to one host core (the oracle is single-threaded; pinning keeps
    the scheduler from moving it). Returns (fn's result, the core used)."""
    try:
        before = os.sched_getaffinity(0)
    except (AttributeError, OSError):
        return fn(), None
    core = max(before)
    os.sched_setaffinity(0, {core})
    try:
        return fn(), core
    finally:
        os.sched_setaffinity(0, before)


def refine_roofline(kname, dL, dR, dmax, R, lr_tol, seconds, traffic=None):
    """Eq. 9-10 as instruction work: the vote window of every pixel that fails the left/right check.
    Per window position (clipped to the image) one load and one test of the voter's validity; per valid
    voter eight more (its colour word, the CIELAB SAD as a four-way absolute difference and a byte sum,
    the two table reads, the product, the shift and the histogram add); per invalid pixel the histogram
    clear and the argmax scan over dmax; per pixel the left/right check (two loads, two tests). Peak:
    the SM's instruction issue rate (4 schedulers x 32 lanes per clock) x SMs x the maximum clock."""
    dL = np.asarray(dL, np.int64)
    dR = np.asarray(dR, np.int64)
    h, w = dL.shape
    ys, xs = np.mgrid[0:h, 0:w]
    xr = xs - dL
    inside = xr >= 0
    partner = dR[ys, np.clip(xr, 0, w - 1)]
    valid = inside & (np.abs(dL - partner) <= lr_tol)
    invalid = ~valid
    # window positions and valid voters per pixel: 2-D box sums over (2R+1)^2 (clipped), by cumulative sums
    def box(a):
        c = np.zeros((h + 1, w + 1), np.int64)
        c[1:, 1:] = a.cumsum(0).cumsum(1)
        y0, y1 = np.clip(np.arange(h) - R, 0, h), np.clip(np.arange(h) + R + 1, 0, h)
        x0, x1 = np.clip(np.arange(w) - R, 0, w), np.clip(np.arange(w) + R + 1, 0, w)
        return c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0]
    positions = int(box(np.ones((h, w), np.int64))[invalid].sum())
    voters = int(box(valid.astype(np.int64))[invalid].sum())
    n_inv = int(invalid.sum())
    ops = 2 * positions + 8 * voters + 2 * dmax * n_inv + 4 * h * w
    peak = SMS * ISSUE_PER_CLK_SM * MAX_SM_MHZ * 1e6 / 1e9
    achieved = ops / seconds / 1e9
    return {"bound": "issue", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "Ginstr/s",
            "frac": achieved / peak, "traffic": traffic, "work_per_launch": ops,
            "peak_basis": f"{SMS} SMs x 4 schedulers x 32 lanes/clk x {MAX_SM_MHZ} MHz",
            "invalid_pixels": n_inv, "window_positions": positions, "valid_voters": voters,
            "note": "lane instructions of Eq. 9-10: 2 per window position, 8 per valid voter, 2 dmax per invalid "
                    "pixel, 4 per pixel for the left/right check; the refinement-word pre-pass is in the stage time"}


def describe_kernel(tuning, nw):
    """(kernel name, source file) of the describe stage the library runs (the dispatch of bsm_describe)."""
    if nw > 8:
        return "describe_wide_kernel", "bsm_long.cu"
    v = tuning.get("describe_variant", 0)
    if v == 2 or (v == 0 and nw == 8):
        return "describe_warp_kernel", "bsm_describe.cu"
    return "describe_kernel", "bsm_describe.cu"


def describe_roofline(kname, pixels, n_bits, seconds, traffic):
    """Eq. 2-7 at the ISA's minimum of 32-bit integer lane operations, 8 per sampling pair: Eq. 3's
    comparison, Eq. 5's two 3-channel SADs (four-way absolute difference + four-way dot product each) and
    their maximum, Eq. 7's comparison with T, and one comparison per pair for Eq. 6's k-th smallest weight
    (a linear-time selection). Peak: the ALU pipe's lanes per clock x SMs x the maximum SM clock."""
    ops = 8 * n_bits * pixels
    peak, basis = alu_peak()
    achieved = ops / seconds / 1e9
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "Gop/s",
            "frac": achieved / peak, "traffic": traffic, "work_per_launch": ops,
            "peak_basis": basis,
            "note": "one view per launch; the T search's bisection and the ballots run on top of the minimum"}


def tensor_roofline(units, n_bits, seconds, traffic):
    """Eq. 8 as a contraction: n multiply-adds per (x, d) and reference view, against the E4M3 dense
    peak (the measured bf16 GEMM rate times the nominal fp8 / bf16 ratio of 2)."""
    flops = 2 * units * 2 * n_bits
    bf16 = measured_peaks().get("bf16_tflops")
    peak, basis = (2 * bf16, "measured bf16 x 2 (nominal fp8/bf16)") if bf16 else (3800.0, "fallback 1.9 PF bf16 x 2")
    achieved = flops / seconds / 1e12
    line = {"bound": "tensor", "kernel": "cost_tc_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "work_per_launch": flops, "peak_basis": basis,
            "note": "one launch covers both reference views; the MMAs also run the window's entering and leaving "
                    "rows and the band around the disparity range"}
    from paper_1402_2020_gb300 import peaks

    f8 = peaks.load_fp8()
    if f8:  # the vendor library's dense E4M3 GEMM rate on this GPU, measured (beside the rule's bf16 x 2): the
        # higher of its single-launch and back-to-back rates
        p8 = max(f8["burst_tflops"], f8["loop_tflops"])
        line["peak_e4m3_gemm_measured"] = {"peak": p8, "frac": achieved / p8,
                                           "basis": "cuBLASLt E4M3 GEMM, 8192^3, " + os.path.relpath(peaks.FP8_SUMMARY, ROOT)}
    return line


def run_pair(args, cfg, world, rank, local, n_bits=N_BITS, window_S=WINDOW_S, sigma=None, agg=AGG, e2e=True,
             cpu_baseline=True):
    """One pair per step through the per-pair C-ABI calls; returns the JSON line (dict)."""
    import torch

    from paper_1402_2020_gb300 import bsm, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, h, dmax = cfg["w"], cfg["h"], cfg["dmax"]
    left, right, gt = synth.stereo_pair(w, h, dmax, cfg["seed"] + rank * 1000, cfg["radiometric"])
    pairs = synth.pair_table(n_bits, window_S, sigma=sigma, seed=PAIR_SEED)
    params = bsm.make_params(pairs, window_S=window_S + (window_S % 2 == 0), agg_window=agg, dmax=dmax,
                             vote_radius=VOTE_R)
    ctx = bsm.bsm_create(params)
    nw = n_bits // 32
    bsm.bsm_set_tuning(ctx, args.cost_rows, args.cost_popc_plain, args.batch_rows, args.cost_variant,
                       args.describe_variant, args.describe_copies)
    if not args.no_autotune and args.cost_rows == 0 and args.cost_variant == 0:
        from paper_1402_2020_gb300 import autotune

        autotune.tune_cost(ctx, n_bits, agg, w, h, dmax)
    stream = torch.cuda.Stream(device=dev)
    s = stream.cuda_stream
    dl = torch.from_numpy(left).to(dev)
    dr = torch.from_numpy(right).to(dev)
    pitch = 3 * w
    BL = torch.empty((h, w, nw), dtype=torch.int32, device=dev)
    PL = torch.empty_like(BL)
    BR = torch.empty_like(BL)
    PR = torch.empty_like(BL)
    dL = torch.empty((h, w), dtype=torch.int32, device=dev)
    dR = torch.empty_like(dL)
    out = torch.empty_like(dL)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    sgm = tuple(int(v) for v in args.sgm.split(",")) if args.sgm else None
    if sgm:  # semi-global aggregation of both views' cost volumes replaces Eq. 1 on the box sums
        cL = torch.empty((h, w, dmax), dtype=torch.int16, device=dev)
        cR = torch.empty_like(cL)
        S = torch.empty((h, w, dmax), dtype=torch.int32, device=dev)
        sL, sR = torch.empty_like(dL), torch.empty_like(dL)

    def step(e=None):
        if e: e[0].record(stream)
        bsm.bsm_describe(ctx, dl, w, h, pitch, BL, PL, s)
        if e: e[1].record(stream)
        bsm.bsm_describe(ctx, dr, w, h, pitch, BR, PR, s)
        if e: e[2].record(stream)
        if sgm:
            bsm.bsm_cost_volumes(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, cL, cR, s)
            if e: e[5].record(stream)  # the two semi-global aggregations, timed apart
            bsm.bsm_sgm(ctx, cL, w, h, dmax, *sgm, S, sL, s)
            bsm.bsm_sgm(ctx, cR, w, h, dmax, *sgm, S, sR, s)
        else:
            bsm.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, None, s)
        if e: e[3].record(stream)
        bsm.bsm_refine(ctx, dl, pitch, *((sL, sR) if sgm else (dL, dR)), w, h, dmax, out, s)
        if e: e[4].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
            flush.zero_()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = Clocks(local)
        clk.start()
        time.sleep(0.3)
        for i in range(args.steps):
            step(ev[i])
            flush.zero_()  # L2 flush between timed steps, outside the step's events
        torch.cuda.synchronize()
        clocks = clk.stop()
    assert bsm.bsm_last_error(ctx) == bsm.BSM_OK
    per = np.array([[ev[i][j].elapsed_time(ev[i][j + 1]) for j in range(4)] for i in range(args.steps)])
    step_ms = per.sum(axis=1)
    t_step = float(step_ms.mean())
    t_step = max_over_ranks([t_step], world, dev)[0]
    units = w * h * dmax
    value = world * units / (t_step * 1e-3) / 1e9

    tuning = bsm.bsm_get_tuning(ctx)
    plan = bsm.bsm_cost_plan(ctx, w, h, dmax)
    kname, kfile, klaunch = plan["name"], plan["source"], plan["launches"]
    bad = bad_pixel_rate(out.cpu().numpy(), gt)
    # rooflines: the cost stage (fused cost/aggregation/WTA, both reference views per launch) and describe
    # (one view per launch); "roofline" is the one of the two that takes more of the step
    t_k2 = float(per[:, 2].mean()) * 1e-3
    word_ops = 2 * units * nw
    achieved = word_ops / t_k2 / 1e9
    peak, popc_basis = popc_peak()
    workload_key = args.config if n_bits == N_BITS else f"{args.config}_n{n_bits}"
    traffic = profile_traffic(kfile, workload_key)
    dname, dfile = describe_kernel(tuning, nw)
    t_desc = float((per[:, 0] + per[:, 1]).mean()) * 1e-3  # two launches
    roof_desc = describe_roofline(dname, w * h, n_bits, t_desc / 2, profile_traffic(dfile, workload_key))
    roof_cost = ({"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                  "unit": "Gpopc/s", "frac": achieved / peak, "traffic": traffic,
                  "work_per_launch": word_ops,
                  "peak_basis": popc_basis}
                 if kname != "cost_tc_kernel" else tensor_roofline(units, n_bits, t_k2, traffic))
    roof_cost["xd_per_s_per_direction"] = units / t_k2  # one launch covers both reference views
    if kname == "cost_tc_kernel":
        # the same launch against the integer-pipe roofline of the popcount formulation of Eq. 8 (one plain
        # POPC per masked word), the bound the popcount kernels are held to
        roof_cost["popc_equivalent"] = {"achieved": achieved, "peak": peak, "unit": "Gpopc/s",
                                        "frac": achieved / peak}
    describe_dominant = t_desc > t_k2
    if kname == "cost_tc_kernel" and not sgm and args.cost_variant == 0:
        # the popcount formulation of Eq. 8 (the two-column kernel) on the same planes, timed apart, against
        # its own integer roofline: the design the tensor-core kernel replaced, reported beside it
        saved = bsm.bsm_get_tuning(ctx)
        try:
            bsm.bsm_set_tuning(ctx, 0, 0, saved["batch_rows"], 2, saved["describe_variant"], saved["describe_copies"])
            ep = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            with torch.cuda.stream(stream):
                for _ in range(2):
                    bsm.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, None, s)
                reps = 5
                ep[0].record(stream)
                for _ in range(reps):
                    bsm.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, None, s)
                ep[1].record(stream)
                torch.cuda.synchronize()
            t_pc = ep[0].elapsed_time(ep[1]) * 1e-3 / reps
            pplan = bsm.bsm_cost_plan(ctx, w, h, dmax)
            pk, pname = pplan["name"], pplan["source"]
            roof_cost["popcount_kernel"] = {
                "bound": "alu", "kernel": pk, "achieved": word_ops / t_pc / 1e9, "peak": peak, "unit": "Gpopc/s",
                "frac": word_ops / t_pc / 1e9 / peak, "stage_ms": t_pc * 1e3,
                "traffic": profile_traffic(pname, workload_key), "peak_basis": popc_basis,
                "note": "the two-column popcount kernel timed on the same planes (not part of the step)"}
        finally:
            bsm.bsm_set_tuning(ctx, saved["cost_rows"], saved["cost_popc_plain"], saved["batch_rows"],
                               saved["cost_variant"], saved["describe_variant"], saved["describe_copies"])
            with torch.cuda.stream(stream):  # the maps of the last timed step again, from the step's own kernel
                bsm.bsm_cost_aggregate_wta(ctx, BL, PL, BR, PR, w, h, dmax, dL, dR, None, s)
            torch.cuda.synchronize()
    rname = "refine_kernel"
    roof_ref = None
    if not sgm:
        roof_ref = refine_roofline(rname, dL.cpu().numpy(), dR.cpu().numpy(), dmax, VOTE_R, 1,
                                   float(per[:, 3].mean()) * 1e-3, profile_traffic("bsm_refine.cu", workload_key))
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg["name"], "n_bits": n_bits, "window_S": window_S, "pair_sigma": sigma,
                   "agg_window": agg, "mask_rank": n_bits // 4, "vote_radius": VOTE_R,
                   "parallelism": f"replicas x{world}",
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "stage_ms": {"describe_left": float(per[:, 0].mean()), "describe_right": float(per[:, 1].mean()),
                     ("cost_volumes_and_sgm" if sgm else "cost_aggregate_wta"): float(per[:, 2].mean()),
                     "refine": float(per[:, 3].mean())},
        "pairs_per_s": world / (t_step * 1e-3),
        "bad_pixel_rate": bad,  # |d - d_gt| > 1 against the generator's ground truth, rank 0's pair
        # colour pre-pass + describe per view, the cost stage's kernels, the refinement-word pass, the block
        # ordering and refine
        "gpu_launches": (4 + klaunch + 3 + (2 * sgm[2] if sgm else 0)) * args.steps,
        "roofline": roof_desc if describe_dominant else roof_cost,
        ("roofline_cost" if describe_dominant else "roofline_describe"): roof_cost if describe_dominant else roof_desc,
        "clocks": clocks,
        "tuning": tuning,
        "cost_plan": plan,
    }
    if sgm:
        line["config"]["sgm"] = {"P1": sgm[0], "P2": sgm[1], "paths": sgm[2]}
        t_sgm = float(np.mean([ev[i][5].elapsed_time(ev[i][3]) for i in range(args.steps)])) * 1e-3
        line["stage_ms"]["sgm_both_views"] = t_sgm * 1e3
        if n_bits * agg * agg + sgm[1] < 65536:
            # concurrent schedule, per (x, d) and view: the maximum (2 B), every direction's cost read and
            # 16-bit path cost written (4 B), the path costs read back (2 B each) and S written (4 B)
            bpx = 2 + 6 * sgm[2] + 4
            hbm = measured_peaks().get("hbm_gbs") or 6800.0
            achieved = 2 * units * bpx / t_sgm / 1e9
            line["roofline_sgm"] = {"bound": "hbm", "kernel": "sgm_path_kernel + sgm_sum_kernel", "achieved": achieved,
                                    "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                                    "work_per_launch": 2 * units * bpx,
                                    "peak_basis": "measured copy bandwidth" if measured_peaks().get("hbm_gbs")
                                    else "fallback 6.8 TB/s",
                                    "note": f"both views' aggregations, {bpx} B per (x, d) and view"}
        # the cost stage also holds both views' semi-global aggregation, so it has no cost roofline of its
        # own; the aggregation's roofline is the headline one where it takes more of the step than describe
        if "roofline_sgm" in line and t_sgm > t_desc:
            line["roofline"] = line["roofline_sgm"]
        else:
            line["roofline"] = roof_desc if describe_dominant else None
        line.pop("roofline_cost", None)
    if e2e and not sgm:
        # end to end through the host-buffer C-ABI call (H2D of both views and D2H of the map inside)
        hl = torch.from_numpy(left).pin_memory()
        hr = torch.from_numpy(right).pin_memory()
        ho = torch.empty((h, w), dtype=torch.int32).pin_memory()
        for _ in range(2):
            bsm.bsm_match_host(ctx, hl.data_ptr(), hr.data_ptr(), w, h, pitch, dmax, ho.data_ptr(), s)
        e2e_t = []
        for _ in range(max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bsm.bsm_match_host(ctx, hl.data_ptr(), hr.data_ptr(), w, h, pitch, dmax, ho.data_ptr(), s)
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = float(np.mean(e2e_t))
        e2e_s = max_over_ranks([e2e_s], world, dev)[0]
        line["e2e"] = {"value": world * units / e2e_s / 1e9, "unit": METRIC, "h2d_bytes_per_step": 2 * h * pitch,
                       "d2h_bytes_per_step": 4 * w * h, "ms_per_step": e2e_s * 1e3}
    if roof_ref is not None:
        line["roofline_refine"] = roof_ref
    if cpu_baseline and rank == 0 and world == 1 and not args.no_cpu_baseline:
        (dt, u), core = pinned_to_one_core(lambda: oracle_sample(cfg, 32))
        nproc, model = host_cpu()
        line["cpu_baseline"] = {"value": u / dt / 1e9, "unit": METRIC, "cores": 1, "kind": "oracle",
                                "sample": f"{w}x32 row band of the workload (rows {h // 2 - 16}..{h // 2 + 15}), whole "
                                          f"oracle pipeline, single thread pinned to host core {core}",
                                "seconds": dt, "nproc": nproc, "cpu_model": model}
    bsm.bsm_destroy(ctx)
    return line


SWEEP_N = (32, 64, 128, 256, 512, 1024, 2048, 4096)


def bad_pixel_rate(disp, gt, tol=1):
    """Share of pixels whose disparity is off the generator's ground truth by more than tol, over the
    pixels whose true match lies inside the right view."""
    disp = np.asarray(disp)
    x = np.arange(gt.shape[1])[None, :]
    m = x - gt >= 0
    return float((np.abs(disp.astype(np.int64) - gt)[m] > tol).mean())


MASK_NAMES = {0: "BSM mask (Eq. 8)", 1: "no mask (Eq. 4)", 2: "both views' masks"}
EXPOSURE = ((0.5, 0.7), (0.5, 1.0), (0.5, 1.4), (1.0, 0.7), (1.0, 1.0), (1.0, 1.4), (2.0, 0.7), (2.0, 1.0),
            (2.0, 1.4))  # (gain, gamma) of the right view: a 3 x 3 exposure / illumination design


def run_quality(args, cfg, world, rank, local):
    """Disparity error against the generator's ground truth (synthetic stand-ins for the paper's
    Middlebury evaluation): the mask ablation (Eq. 8's mask, no mask as in Eq. 4, both views' masks) for
    window 1 and 5, and the same three under a 3 x 3 radiometric design applied to the right view."""
    import torch

    from paper_1402_2020_gb300 import bsm, synth

    if rank != 0:
        return
    torch.cuda.set_device(local)
    w, h, dmax = cfg["w"], cfg["h"], cfg["dmax"]
    seeds = range(cfg["seed"], cfg["seed"] + 3)
    views = {s: synth.stereo_pair(w, h, dmax, s) for s in seeds}
    # this library's default descriptor, and the paper's (n = 4096, S = 26, sigma = 4) with a 3 x 3 box
    settings = {"n=256, S=31": (256, 31, None, AGG), "n=4096, S=26, sigma=4": (4096, 26, 4.0, 3)}

    def evaluate(setting, mode, agg, transform=None, sgm=None):
        n, S, sigma, _ = settings[setting]
        pairs = synth.pair_table(n, S, sigma=sigma, seed=PAIR_SEED)
        m = bsm.Matcher(pairs, window_S=S + (S % 2 == 0), agg_window=agg, dmax=dmax, vote_radius=VOTE_R,
                        mask_mode=mode)
        rates = []
        for s in seeds:
            left, right, gt = views[s]
            if transform is not None:
                right = transform(right)
            dl, dr = torch.from_numpy(left).cuda(), torch.from_numpy(np.ascontiguousarray(right)).cuda()
            out = m.match(dl, dr, dmax) if sgm is None else m.match_sgm(dl, dr, dmax, *sgm)
            rates.append(bad_pixel_rate(out.cpu().numpy(), gt))
        m.close()
        return float(np.mean(rates))

    table, radio = {}, {}
    for setting, (_, _, _, agg_box) in settings.items():
        for mode in (0, 1, 2):
            for agg in (1, agg_box):
                table[f"{setting}: {MASK_NAMES[mode]}, window {agg}"] = evaluate(setting, mode, agg)
            if setting.startswith("n=256"):
                for agg in (1, agg_box):
                    for P1, P2 in ((2, 8), (4, 32)):
                        P1w, P2w = P1 * agg * agg, P2 * agg * agg
                        table[f"{setting}: {MASK_NAMES[mode]}, window {agg}, SGM 8 paths P1={P1w} P2={P2w}"] = \
                            evaluate(setting, mode, agg, sgm=(P1w, P2w, 8))
            radio[f"{setting}: {MASK_NAMES[mode]}, window {agg_box}"] = {
                f"gain {g} gamma {gm}": evaluate(setting, mode, agg_box,
                                                 lambda r, g=g, gm=gm: synth.radiometric_fixed(r, g, gm))
                for g, gm in EXPOSURE}
    line = {"metric": "bad-pixel rate (|d - d_gt| > 1)", "unit": "fraction", "higher_is_better": False,
            "data": "synthetic", "config": {"workload": cfg["name"], "settings": list(settings),
                                            "seeds": list(seeds), "vote_radius": VOTE_R},
            "mask_ablation": table, "radiometric_3x3": radio}
    print(json.dumps(line), flush=True)


def run_sweep_n(args, cfg, world, rank, local):
    """Speed against descriptor length (the speed half of Fig. 3b): the paper's pair distribution
    (S = 26, sigma = 4), a 3x3 box (n * 3^2 fits the 16-bit cost for every n), one line per n."""
    agg = 3
    for n in SWEEP_N:
        line = run_pair(args, cfg, world, rank, local, n_bits=n, window_S=26, sigma=4.0, agg=agg, e2e=False,
                        cpu_baseline=False)
        line["sweep"] = "descriptor length n (Fig. 3b)"
        if rank == 0:
            print(json.dumps(line), flush=True)


def run_default(args, world, rank, local):
    """The headline: the 3840 x 2160 pair (the largest single-GPU configuration, the one the fused cost
    kernel's roofline is judged on), with the batched (c3) and served (c5) objects in the same line."""
    args.config = "c4"
    line = run_pair(args, CONFIGS["c4"], world, rank, local)
    if not args.no_batched:
        b = run_batch(args, CONFIGS["c3"], world, rank, local)
        b["workload"] = CONFIGS["c3"]["name"]
        line["batched"] = b
    if not args.no_served:
        sv = run_serving(args, CONFIGS["c5"], world, rank, local)
        sv["workload"] = CONFIGS["c5"]["name"]
        line["served"] = sv
    return line


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, CONFIGS[args.config or "c4"], world, rank)
        return
    cfg = CONFIGS.get(args.config)
    if not args.config and not (args.sweep_n or args.quality):
        line = run_default(args, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    elif args.config in ("c3", "c5"):
        line = (run_batch if args.config == "c3" else run_serving)(args, cfg, world, rank, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
    else:
        if not args.config:
            args.config, cfg = "c2", CONFIGS["c2"]
        if args.sweep_n:
            run_sweep_n(args, cfg, world, rank, local)
        elif args.quality:
            run_quality(args, cfg, world, rank, local)
        else:
            agg = AGG if args.n_bits * AGG * AGG <= 65535 else 3  # the 16-bit aggregated cost bounds n * W^2
            line = run_pair(args, cfg, world, rank, local, n_bits=args.n_bits, agg=agg)
            if rank == 0:
                print(json.dumps(line), flush=True)
    if world > 1:
        torch_dist_done()


if __name__ == "__main__":
    main()
