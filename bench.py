"""Benchmark of the MergeShuffle hot path on GB300 (one JSON line on rank 0).

Workload (default "scale"): one step = perm(n = 2^30) of the uint32 identity plus a shuffle of
n = 300,000,017 16-byte records {u32 key = index, 12-byte splitmix64 payload}, seed 7, both in
HBM before the timed region. value = elements permuted per second over both calls (Gelem/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (single-threaded C restatement of the paper) on a bounded
sample of the same workload. Under torchrun (N > 1) each rank runs an independent replica of
the workload (the path has no cross-GPU step); the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_PERM = 1 << 30
N_REC = 300_000_017
SEED = 7
DEFAULT_B = {"perm": 0, "rec": 0}  # 0: the autotuner's table chooses (reported as resolved)
SCALE_WORKLOAD = ("plain MergeShuffle at scale: perm of n=2^30 uint32 identity + shuffle of "
                  "n=300000017 16-byte records {u32 key, 12-byte splitmix64 payload}, seed 7")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--B-perm", type=int, default=DEFAULT_B["perm"])
    ap.add_argument("--B-rec", type=int, default=DEFAULT_B["rec"])
    ap.add_argument("--tile-bytes", type=int, default=0)
    ap.add_argument("--fuse-depth", type=int, default=-1,
                    help="merge levels fused into the base-block kernel (-1: autotuned)")
    ap.add_argument("--fuse-depth-perm", type=int, default=None,
                    help="as --fuse-depth, for the perm only")
    ap.add_argument("--fuse-depth-rec", type=int, default=None,
                    help="as --fuse-depth, for the records only")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--overlap", choices=["none", "equal", "perm-high", "rec-high"],
                    default="none",
                    help="device step: run the perm and the records one after the other on one "
                         "stream (none), or on two streams at the given priorities")
    ap.add_argument("--serve-window", type=float, default=0.25,
                    help="seconds of 20k/s arrivals in the serving overload run")
    ap.add_argument("--serve-sub-rate", type=float, default=1500.0)
    ap.add_argument("--serve-sub-window", type=float, default=2.0)
    ap.add_argument("--serve-inflight", type=int, default=4,
                    help="launches the server keeps on the GPU at once (one stream each)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="scale workload only: skip the batched, batched-large and serving "
                         "sub-objects of the default line")
    ap.add_argument("--workload", choices=["scale", "batched", "batched-large", "serve", "rs",
                                           "variants"],
                    default="scale",
                    help="rs: the Rao-Sandelius perm alone; variants: the literal, FDR and "
                         "balanced-word perms and the Table 1 bit counts alone")
    ap.add_argument("--flags-perm", type=lambda x: int(x, 0), default=0,
                    help="MS_FLAG_* bits added to the perm's resolved flags (e.g. 0x100: fused "
                         "pairs of 4-byte levels)")
    ap.add_argument("--flags-rec", type=lambda x: int(x, 0), default=0,
                    help="MS_FLAG_* bits added to the records' resolved flags")
    ap.add_argument("--unflags-perm", type=lambda x: int(x, 0), default=0,
                    help="MS_FLAG_* bits removed from the perm's resolved flags (e.g. 0x80, "
                         "the table's one-pass-a-level choice at 2^30)")
    ap.add_argument("--small", action="store_true",
                    help="profiling case: perm 2^26 + 2^24+17 records (inputs still above L2)")
    return ap.parse_args()


# ------------------------------------------------------------------ distributed plumbing -----
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks ------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.reader = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        loaded = sorted(sm)
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm -----------------
def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# DRAM bytes (read + written) per element of one gather launch, from an ncu capture of the
# gather kernels on a smaller case with inputs above L2 (perm 2^26: the staged gather of 4-byte
# elements; records 2^24 + 17: the 16-byte gather), scaled to a full launch by the elements it
# processes
GATHER_TRAFFIC_PER_ELEM = {4: 7.182, 16: 28.71}


# the cutoffs the built-in tuning table resolves the scale workload to (the GPU arm checks it;
# the reference arm uses them without loading the CUDA library)
TUNED_B = {"perm": 512, "rec": 572}

# kernel classes whose CUDA-event spans measure their own duration (launched in order on the
# caller's stream), and those launched on the paired plan stream, whose spans also cover the time
# they wait for SMs held by the data pass they overlap
DATA_STREAM_KINDS = ("leaf", "gather", "pair_gather", "patch_read", "patch_write",
                     "tail_sequential", "local")
PLAN_STREAM_KINDS = ("count", "scan", "kscan", "hash_clear", "tail_insert", "tail_resolve",
                     "exceptions")


def perm_bytes(n: int, passes: int) -> int:
    """Algorithmic HBM bytes of a perm: its first pass only writes (4n), every later pass reads
    and writes the array (2 * 4n)."""
    return (2 * passes - 1) * 4 * n if passes > 0 else 0


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_1508_03167_gb300 as ms
    from paper_1508_03167_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    n_perm = (1 << 26) if args.small else N_PERM
    n_rec = (1 << 24) + 17 if args.small else N_REC
    seed = SEED + rank
    # B = 0 resolves through the autotuner's table; the resolved parameters define the result
    fd_perm = args.fuse_depth if args.fuse_depth_perm is None else args.fuse_depth_perm
    fd_rec = args.fuse_depth if args.fuse_depth_rec is None else args.fuse_depth_rec
    p_perm = ms.resolve(n_perm, 4, B=args.B_perm, fuse_depth=fd_perm, tile_bytes=args.tile_bytes)
    p_rec = ms.resolve(n_rec, 16, B=args.B_rec, fuse_depth=fd_rec, tile_bytes=args.tile_bytes)
    p_perm.flags = (p_perm.flags | args.flags_perm) & ~args.unflags_perm
    p_rec.flags |= args.flags_rec
    prof_perm = ms.params(p_perm.B, p_perm.fuse_depth, p_perm.flags | ms.MS_FLAG_PROFILE,
                          p_perm.tile_bytes)
    prof_rec = ms.params(p_rec.B, p_rec.fuse_depth, p_rec.flags | ms.MS_FLAG_PROFILE,
                         p_rec.tile_bytes)
    # (the perm's plan, not the 4-byte shuffle's: a shuffle whose first pass is the tile kernel
    # may fuse one level less so that this pass does not run in place)
    plan_perm = ms.ms_plan_info(n_perm, 4, ms.params(p_perm.B, p_perm.fuse_depth,
                                                     p_perm.flags | ms.MS_FLAG_PERM,
                                                     p_perm.tile_bytes))
    plan_rec = ms.ms_plan_info(n_rec, 16, p_rec)

    out = torch.empty(n_perm, dtype=torch.int32, device=dev)
    ws_perm = torch.empty(ms.ms_workspace_bytes(n_perm, 4, p_perm), dtype=torch.uint8, device=dev)
    rec_host = torch.from_numpy(inputs.records16(n_rec))
    rec = rec_host.to(dev)
    ws_rec = torch.empty(ms.ms_workspace_bytes(n_rec, 16, p_rec), dtype=torch.uint8, device=dev)

    # the two calls are independent; with --overlap the records run on a second stream, forked
    # from and joined back into the timed stream every step, so that one call's latency-bound
    # base-block pass can overlap the other's memory-bound level passes
    s_perm, s_rec = sh, sh
    fork = join = None
    if args.overlap != "none":
        prio = {"equal": (0, 0), "perm-high": (-1, 0), "rec-high": (0, -1)}[args.overlap]
        st_perm = torch.cuda.Stream(device=dev, priority=prio[0])
        st_rec = torch.cuda.Stream(device=dev, priority=prio[1])
        s_perm, s_rec = st_perm.cuda_stream, st_rec.cuda_stream
        fork = torch.cuda.Event()
        join = [torch.cuda.Event(), torch.cuda.Event()]

    def step(profiled: bool, mid=None):
        if fork is not None:
            fork.record(stream)
            st_perm.wait_event(fork)
            st_rec.wait_event(fork)
        st = ms.ms_perm(out.data_ptr(), n_perm, seed, ws_perm.data_ptr(), ws_perm.numel(),
                        prof_perm if profiled else p_perm, s_perm)
        if st != ms.MS_OK:
            raise ms.MsError(st, "ms_perm")
        if mid is not None:
            mid.record(stream)
        st = ms.ms_shuffle(rec.data_ptr(), n_rec, 16, seed, ws_rec.data_ptr(), ws_rec.numel(),
                           prof_rec if profiled else p_rec, s_rec)
        if st != ms.MS_OK:
            raise ms.MsError(st, "ms_shuffle")
        if fork is not None:
            join[0].record(st_perm)
            join[1].record(st_rec)
            stream.wait_event(join[0])
            stream.wait_event(join[1])

    for _ in range(args.warmup):
        step(False)
    step(True)  # the profiled variant's first call (events created outside the timed regions)
    torch.cuda.synchronize(dev)
    ms.profile(reset=True)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # timed region 1 (the headline): the plain calls, an event between the perm and the records
    # of every step (on one stream: the perm's and the records' shares of the step)
    barrier(world)
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        evs[k][0].record(stream)
        step(False, mid=evs[k][1] if fork is None else None)
        evs[k][2].record(stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    t_ms = e0.elapsed_time(e1) / args.steps
    t_perm_ms = t_rec_ms = None
    if fork is None:
        t_perm_ms = sum(a.elapsed_time(b) for a, b, _ in evs) / args.steps
        t_rec_ms = sum(b.elapsed_time(c) for _, b, c in evs) / args.steps
    t_ms = allreduce_max(t_ms, world)
    # timed region 2: the same steps with an event pair around every kernel (MS_FLAG_PROFILE),
    # for the per-kernel figures; its step time against region 1 is the profiling overhead
    torch.cuda.synchronize(dev)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        step(True)
    e3.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_prof_ms = e2.elapsed_time(e3) / args.steps
    prof = ms.profile(reset=True)

    elems = n_perm + n_rec
    value = world * elems / (t_ms * 1e-3) / 1e9
    peaks = measured_peaks()
    bw = peaks["hbm_gbs"]

    # roofline of the dominant kernel, the streaming gather of a global merge level (one
    # launch per unfused level): algorithmic bytes per launch = read n*w + write n*w. Fused
    # pairs of levels (a pair_gather launch each, also one read and one write of the array) and
    # the tile kernel (first pass: the perm only writes 4n, a shuffle reads and writes n*w) are
    # reported beside it. Kernel times: CUDA events around each launch on the caller's stream.
    g = prof.get("gather", {"ms": 0.0, "launches": 0})
    pg = prof.get("pair_gather", {"ms": 0.0, "launches": 0})
    lf = prof.get("leaf", {"ms": 0.0, "launches": 0})
    single_perm = plan_perm.global_levels - 2 * plan_perm.fused_pairs
    single_rec = plan_rec.global_levels - 2 * plan_rec.fused_pairs
    gather_bytes = args.steps * (single_perm * 2 * n_perm * 4 + single_rec * 2 * n_rec * 16)
    pair_bytes = args.steps * (plan_perm.fused_pairs * 2 * n_perm * 4 +
                               plan_rec.fused_pairs * 2 * n_rec * 16)
    tile_bytes = args.steps * (4 * n_perm + 2 * 16 * n_rec)
    achieved = gather_bytes / (g["ms"] * 1e-3) / 1e9 if g["ms"] > 0 else 0.0
    nlaunch = single_perm + single_rec
    traffic = ((single_perm * GATHER_TRAFFIC_PER_ELEM[4] * n_perm +
                single_rec * GATHER_TRAFFIC_PER_ELEM[16] * n_rec) / nlaunch) if nlaunch else None
    path_perm = perm_bytes(n_perm, plan_perm.passes)
    path_rec = plan_rec.passes * 2 * n_rec * 16
    path_perm_unfused = perm_bytes(n_perm, plan_perm.passes + plan_perm.fused_pairs)
    path_rec_unfused = (plan_rec.passes + plan_rec.fused_pairs) * 2 * n_rec * 16

    def frac(nbytes, ms_):
        return round(nbytes / 1e9 / (ms_ * 1e-3) / bw, 4) if ms_ else None

    roofline = {
        "bound": "hbm",
        "kernel": "gather (HBM merge level)",
        "achieved": round(achieved, 1),
        "peak": bw,
        "peak_source": peaks["source"],
        "unit": "GB/s",
        "frac": round(achieved / bw, 4),
        "traffic": round(traffic) if traffic else None,
        "traffic_note": "bytes per gather launch (dram read+write), ncu on a smaller case "
                        "scaled by elements; the small case leaves ~50 MB of writes in L2",
        "algorithmic_bytes_per_launch": {"perm": 2 * n_perm * 4, "rec": 2 * n_rec * 16},
        "launches_per_step": {"perm": single_perm, "rec": single_rec},
        "avg_launch_ms": round(g["ms"] / max(g["launches"], 1), 4),
        "pair_gather": {
            "launches_per_step": {"perm": plan_perm.fused_pairs, "rec": plan_rec.fused_pairs},
            "achieved_gbs": round(pair_bytes / (pg["ms"] * 1e-3) / 1e9, 1) if pg["ms"] else None,
            "frac": frac(pair_bytes, pg["ms"]),
        },
        "tile": {
            "kernel": "tile kernel (Fisher-Yates and the first d merge levels, one pass)",
            "algorithmic_bytes_per_step": {"perm": 4 * n_perm, "rec": 2 * 16 * n_rec},
            "ms_per_step": round(lf["ms"] / args.steps, 3),
            "achieved_gbs": round(tile_bytes / (lf["ms"] * 1e-3) / 1e9, 1) if lf["ms"] else None,
            "frac": frac(tile_bytes, lf["ms"]),
        },
        # whole path: (algorithmic bytes of all passes / peak) / time; the perm's first pass
        # writes only. "fused" counts a fused pair (and the tile kernel's levels) as one pass,
        # "unfused" every global level as a pass.
        "whole_path_bytes_per_step": {"perm": path_perm, "rec": path_rec},
        "whole_path_frac": frac(path_perm + path_rec, t_ms),
        "whole_path_frac_unfused": frac(path_perm_unfused + path_rec_unfused, t_ms),
        "whole_path_frac_perm": frac(path_perm, t_perm_ms),
        "whole_path_frac_rec": frac(path_rec, t_rec_ms),
    }
    kernel_ms = {k: round(prof[k]["ms"] / args.steps, 3) for k in DATA_STREAM_KINDS
                 if k in prof and prof[k]["launches"]}
    plan_ms = {k: round(prof[k]["ms"] / args.steps, 3) for k in PLAN_STREAM_KINDS
               if k in prof and prof[k]["launches"]}
    launches = args.steps * (plan_perm.kernel_launches + plan_rec.kernel_launches)
    # end to end through the host-buffer entry points: H2D of the input, the shuffle, D2H of
    # the result, every step
    e2e = None
    if not args.no_e2e:
        del ws_perm, ws_rec
        torch.cuda.empty_cache()
        hp = torch.empty(n_perm, dtype=torch.int32, pin_memory=True)
        hr = torch.empty((n_rec, 4), dtype=torch.int32, pin_memory=True)
        hr.copy_(rec_host)
        q_perm = p_perm
        q_rec = p_rec
        wsh_perm = torch.empty(ms.ms_host_workspace_bytes(n_perm, 4, q_perm), dtype=torch.uint8,
                               device=dev)
        wsh_rec = torch.empty(ms.ms_host_workspace_bytes(n_rec, 16, q_rec), dtype=torch.uint8,
                              device=dev)

        # the two calls are independent: issue them from two host threads on two streams, so
        # one's copies overlap the other's kernels (each call synchronises only its own stream).
        # The perm (no input copy) runs at the higher priority and finishes first: its result
        # copy then overlaps the records' kernels, while the records' input copy overlapped the
        # perm's kernels (the copies, ~200 GB/s each way, bound this figure)
        from concurrent.futures import ThreadPoolExecutor

        s_perm = torch.cuda.Stream(device=dev, priority=-1)
        s_rec = torch.cuda.Stream(device=dev, priority=0)
        pool = ThreadPoolExecutor(max_workers=2)

        def call_perm():
            st = ms.ms_perm_host(hp.data_ptr(), n_perm, seed, wsh_perm.data_ptr(),
                                 wsh_perm.numel(), q_perm, s_perm.cuda_stream)
            if st != ms.MS_OK:
                raise ms.MsError(st, "ms_perm_host")

        def call_rec():
            st = ms.ms_shuffle_host(hr.data_ptr(), n_rec, 16, seed, wsh_rec.data_ptr(),
                                    wsh_rec.numel(), q_rec, s_rec.cuda_stream)
            if st != ms.MS_OK:
                raise ms.MsError(st, "ms_shuffle_host")

        def e2e_step():
            fa = pool.submit(call_perm)
            fb = pool.submit(call_rec)
            fa.result()
            fb.result()

        e2e_step()
        k2 = max(2, min(args.steps, 10))
        barrier(world)
        t0 = time.perf_counter()
        each = []
        for _ in range(k2):
            t1 = time.perf_counter()
            e2e_step()
            each.append(round((time.perf_counter() - t1) * 1e3, 1))
        t_e2e = (time.perf_counter() - t0) / k2
        t_e2e = allreduce_max(t_e2e, world)
        pool.shutdown()
        e2e = {"value": round(world * elems / t_e2e / 1e9, 4), "unit": "Gelem/s",
               "h2d_bytes_per_step": n_rec * 16, "d2h_bytes_per_step": n_perm * 4 + n_rec * 16,
               "ms_per_step": round(t_e2e * 1e3, 3), "steps": k2, "ms_each_step": each,
               "how": "ms_perm_host and ms_shuffle_host (pinned host buffers; copies, kernels "
                      "and the stream synchronisation inside each call) issued concurrently "
                      "from two host threads on two streams, the perm's at higher priority"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p_perm.B, p_rec.B)

    # random bits consumed (the paper's Table 1 measure), counted on the GPU outside the timed
    # region: n log2 n + Theta(n) for this method
    import math

    bits = {}
    for tag, n_, B_ in (("perm", n_perm, p_perm.B), ("rec", n_rec, p_rec.B)):
        rb = ms.random_bits(n_, SEED, device=dev, B=B_)
        bits[tag] = {"bits_per_element": round(rb["total_bits"] / n_, 4),
                     "log2_n": round(math.log2(n_), 4),
                     "coin_bits": rb["coin_bits"], "leaf_bits": rb["leaf_bits"],
                     "tail_bits": rb["tail_bits"]}

    line = {
        "metric": "Gelem/s",
        "value": round(value, 4),
        "unit": "Gelem/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_ms, 3),
        "ms_per_step_perm": round(t_perm_ms, 3) if t_perm_ms else None,
        "ms_per_step_rec": round(t_rec_ms, 3) if t_rec_ms else None,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {
            "workload": (SCALE_WORKLOAD if not args.small
                         else "small profiling case: perm 2^26 + 2^24+17 records"),
            "n_perm": n_perm, "n_rec": n_rec, "seed": SEED,
            "B_perm": p_perm.B, "B_rec": p_rec.B,
            "B_source": "autotuner table" if args.B_perm == 0 else "command line",
            "fuse_depth_perm": plan_perm.fuse_depth, "fuse_depth_rec": plan_rec.fuse_depth,
            "passes_perm": plan_perm.passes, "passes_rec": plan_rec.passes,
            "fused_level_pairs_perm": plan_perm.fused_pairs,
            "fused_level_pairs_rec": plan_rec.fused_pairs,
            "l2": "inputs larger than L2 (4.3 GB and 4.8 GB arrays), no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "overlap": args.overlap,
            "timed": "value and ms_per_step: the plain calls; the per-kernel figures come from "
                     "a second timed region of the same steps with a CUDA event pair around "
                     "every kernel (MS_FLAG_PROFILE)",
            "ms_per_step_profiled": round(t_prof_ms, 3),
        },
        "roofline": roofline,
        "kernel_ms_per_step": kernel_ms,
        "plan_stream_event_ms_per_step": plan_ms,
        "plan_stream_note": "the plan kernels run on a second stream beside the data passes; "
                            "their event spans include the time they wait for SMs, so they "
                            "overlap the data-stream figures and do not add up with them",
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "random_bits": bits,
    }
    if not args.small and args.B_perm == 0 and args.B_rec == 0:
        line["config"]["B_matches_reference_arm"] = (p_perm.B == TUNED_B["perm"] and
                                                     p_rec.B == TUNED_B["rec"])
    if world == 1 and not args.small and not args.no_extra:
        # the batched, batched-large and served forms, each against one launch per instance
        # (one request at a time), on the same GPU after the scale workload's buffers are freed
        del out, rec
        if e2e is not None:
            del hp, hr, wsh_perm, wsh_rec  # (the e2e leg already freed ws_perm and ws_rec)
        else:
            del ws_perm, ws_rec
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        ks, kw = max(3, min(args.steps, 10)), 3
        line["batched"] = run_batched(args, large=False, steps=ks, warmup=kw)
        line["batched_large"] = run_batched(args, large=True, steps=ks, warmup=kw)
        line["serve"] = run_serve(args)
        line["rao_sandelius"] = run_rs(args, t_perm_ms)
        line["merge_variants"] = run_literal_fdr(args)
    if rank == 0:
        print(json.dumps(line), flush=True)



# ------------------------------------------------------------------ CPU oracle --------------
def cpu_baseline(B_perm: int, B_rec: int) -> dict:
    """The oracle as it stands on one host core, on a bounded sample of the workload (the same
    element mix as the GPU step, 1/16 of its perm and 1/18 of its records: about 10-30 s)."""
    import oracle
    from paper_1508_03167_gb300 import inputs

    n1 = 1 << 26
    n2 = 1 << 24
    rec = inputs.records16(n2)
    t0 = time.perf_counter()
    oracle.perm(n1, SEED, B_perm)
    oracle.shuffle(rec, SEED, B_rec)
    dt = time.perf_counter() - t0
    return {"value": round((n1 + n2) / dt / 1e9, 6), "unit": "Gelem/s", "cores": 1,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"perm(2^26) u32 + shuffle(2^24) 16-byte records, B={B_perm}/{B_rec}, "
                      f"single-threaded C oracle, {dt:.1f} s"}


def run_reference(args, world, rank):
    """--impl reference: the oracle timed on bounded samples of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_1508_03167_gb300 import inputs

    n1 = 1 << 21
    n2 = 1 << 19
    rec = inputs.records16(n2)
    # the B the GPU arm runs the full-size workload with (the tuning table's choice, which the
    # GPU arm checks); this arm never loads the CUDA library
    B_perm = args.B_perm or TUNED_B["perm"]
    B_rec = args.B_rec or TUNED_B["rec"]

    def step():
        oracle.perm(n1, SEED, B_perm)
        oracle.shuffle(rec, SEED, B_rec)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = (n1 + n2) / dt / 1e9
    sample = (f"per step: perm(2^21) u32 + shuffle(2^19) 16-byte records of the same workload, "
              f"B={B_perm}/{B_rec}, single-threaded C oracle")
    line = {
        "impl": "reference",
        "metric": "Gelem/s",
        "value": round(value, 6),
        "unit": "Gelem/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        # the GPU arm's workload; each timed step is the bounded sample stated below
        "config": {"workload": SCALE_WORKLOAD, "n_perm": N_PERM, "n_rec": N_REC, "seed": SEED,
                   "B_perm": B_perm, "B_rec": B_rec,
                   "sample": {"n_perm": n1, "n_rec": n2}},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gelem/s", "cores": 1,
                         "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed_graph(torch, fn, steps, warmup):
    """Capture fn() (stream work only) into a CUDA graph and time `steps` replays."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fn(s)  # eager run: kernel attributes are set outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn(s)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_batched(args, large: bool, steps: int | None = None, warmup: int | None = None) -> dict:
    """4096 perm(n_i), n_i log-uniform in [2^6, 2^20], seed_i = 1 + i (batched), or 64 shuffles
    of uint64 arrays, n_i uniform in [10^6, 10^8] non-power-of-two (batched-large); one prepared
    batch replayed from a CUDA graph, against one launch sequence per instance."""
    import torch

    import paper_1508_03167_gb300 as ms
    from paper_1508_03167_gb300 import inputs

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    if large:
        sizes = [int(x) for x in inputs.batch_sizes_uniform(64, 10**6, 10**8)]
        w, B, flags = 8, args.B_rec, 0
        bufs = [inputs.values_u64_torch(n, i).view(torch.int64) for i, n in enumerate(sizes)]
        base_seed = 1
    else:
        sizes = [int(x) for x in inputs.batch_sizes_log_uniform(4096, 6, 20)]
        w, B, flags = 4, args.B_perm, ms.MS_FLAG_PERM
        bufs = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
        base_seed = 1
    # one B for the batch (B = 0: the autotuner's batch row); the per-launch baseline uses the
    # same B, so both produce the same permutations
    B = ms.resolve_batch(sizes, w, B=B, flags=flags).B
    p = ms.params(B=B, flags=flags)
    ptrs = [b.data_ptr() for b in bufs]
    nbytes = ms.ms_batch_workspace_bytes(sizes, w, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    total = sum(sizes)

    def prep(s):
        assert ms.ms_batch_prepare(ptrs, sizes, w, None, base_seed, ws.data_ptr(), nbytes, p,
                                   s.cuda_stream) == ms.MS_OK

    def run(s):
        assert ms.ms_batch_run(ptrs, sizes, w, None, base_seed, ws.data_ptr(), nbytes, p,
                               s.cuda_stream) == ms.MS_OK

    s0 = torch.cuda.Stream()
    with torch.cuda.stream(s0):
        prep(s0)
    s0.synchronize()
    t_batch = _timed_graph(torch, run, steps, warmup)
    # one launch sequence per instance (the same library, no batching)
    q = ms.params(B=B)
    wss = torch.empty(max(ms.ms_workspace_bytes(n, w, q) for n in sizes), dtype=torch.uint8,
                      device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def per_launch():
        for i, n in enumerate(sizes):
            if large:
                rc = ms.ms_shuffle(ptrs[i], n, w, base_seed + i, wss.data_ptr(), wss.numel(), q,
                                   st)
            else:
                rc = ms.ms_perm(ptrs[i], n, base_seed + i, wss.data_ptr(), wss.numel(), q, st)
            assert rc == ms.MS_OK

    per_launch()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    per_launch()
    e1.record()
    torch.cuda.synchronize()
    t_single = max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3)
    # roofline: algorithmic bytes of the batch over its time and the measured copy peak; the
    # one-pass bound moves each instance once (a perm only writes it), the pass-counted figure
    # charges every instance the HBM passes of its single-call plan at the batch's B
    bw = measured_peaks()["hbm_gbs"]
    one_pass = sum((4 * n) if not large else (2 * w * n) for n in sizes)
    passes = 0
    for n in sizes:
        pl = ms.ms_plan_info(n, w, ms.params(B=B, flags=flags))
        passes += perm_bytes(n, pl.passes) if not large else pl.passes * 2 * w * n
    del wss, ws, bufs
    torch.cuda.empty_cache()
    return {
        "metric": "Gelem/s", "value": round(total / (t_batch * 1e-3) / 1e9, 4),
        "unit": "Gelem/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": round(t_batch, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32" if not large else "u64", "data": "synthetic",
        "config": {
            "workload": ("batched: 4096 perm(n_i) uint32, n_i log-uniform in [2^6, 2^20], "
                         "seed_i = 1 + i" if not large else
                         "batched large: 64 shuffles of uint64 arrays (splitmix64 values), "
                         "n_i uniform in [1e6, 1e8] non-power-of-two, seed_i = 1 + i"),
            "instances": len(sizes), "elements": total, "B": B,
            "graph": "prepared batch replayed from one CUDA graph",
            "device_bytes": int(nbytes + sum(n * w for n in sizes)),
        },
        "roofline": {
            "bound": "hbm", "peak": bw, "unit": "GB/s",
            "one_pass_bytes": one_pass,
            "one_pass_frac": round(one_pass / 1e9 / (t_batch * 1e-3) / bw, 4),
            "passes_bytes": passes,
            "passes_frac": round(passes / 1e9 / (t_batch * 1e-3) / bw, 4),
        },
        "per_launch": {"ms": round(t_single, 3),
                       "gelem_per_s": round(total / (t_single * 1e-3) / 1e9, 4),
                       "how": "one ms_perm / ms_shuffle launch sequence per instance"},
        "speedup_vs_per_launch": round(t_single / t_batch, 2),
    }


def run_rs(args, t_ms_mergeshuffle=None, steps: int = 5, warmup: int = 2) -> dict:
    """The comparison workload: the Rao-Sandelius splitting process (Fisher-Yates cutoff B)
    filling a perm of 2^30 uint32 with seed 7 and B = 512 (the MergeShuffle perm's tuned cutoff),
    timed like the scale step's perm, beside that perm's own time."""
    import torch

    import paper_1508_03167_gb300 as ms

    n = (1 << 26) if args.small else N_PERM
    B = TUNED_B["perm"]
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    nbytes = ms.ms_rs_workspace_bytes(n, 4, B)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()

    def call():
        st = ms.ms_rs_perm(out.data_ptr(), n, SEED, B, ws.data_ptr(), nbytes, s.cuda_stream)
        if st != ms.MS_OK:
            raise ms.MsError(st, "ms_rs_perm")

    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record(s)
        call()  # (the call waits once for its stream: the host reads the unfinished count)
        b.record(s)
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) / steps
    c = 0
    while (n >> c) > B:
        c += 1
    # the library plans c + 1 levels, made odd by one more unless the Fisher-Yates pass runs in
    # place (4-byte rows, B <= 512)
    levels = c + 1 + ((c + 1) % 2 == 0 and B > 512)
    # algorithmic bytes: the first split level only writes (4n), every other split level and the
    # Fisher-Yates pass read and write the array
    nb = 4 * n + (levels - 1) * 8 * n + 8 * n
    bw = measured_peaks()["hbm_gbs"]
    del out, ws
    torch.cuda.empty_cache()
    return {
        "metric": "Gelem/s", "value": round(n / (t * 1e-3) / 1e9, 4), "unit": "Gelem/s",
        "ms_per_call": round(t, 3), "steps": steps, "warmup": warmup, "dtype": "u32",
        "config": {"workload": f"Rao-Sandelius splitting process, perm of n={n} uint32, seed "
                               f"{SEED}, Fisher-Yates cutoff B={B}", "n": n, "B": B,
                   "split_levels_planned": levels},
        "roofline": {"bound": "hbm", "bytes_per_call": nb, "peak": bw, "unit": "GB/s",
                     "achieved": round(nb / 1e9 / (t * 1e-3), 1),
                     "frac": round(nb / 1e9 / (t * 1e-3) / bw, 4)},
        "mergeshuffle_perm_ms": round(t_ms_mergeshuffle, 3) if t_ms_mergeshuffle else None,
        "mergeshuffle_speedup": (round(t / t_ms_mergeshuffle, 3) if t_ms_mergeshuffle else None),
    }


def run_literal_fdr(args, steps: int = 3, warmup: int = 1) -> dict:
    """Algorithm 3 as printed (MS_FLAG_LITERAL), Fast Dice Roller draws (MS_FLAG_FDR) and merges
    driven by a balanced word (MS_FLAG_BALANCED) on the scale workload's perm (2^30, seed 7,
    B = 512), timed beside the default plan with the same forced shape (fuse_depth 0, one global
    pass per level); and Table 1's measure, the random bits consumed, counted on the GPU for
    n = 10^5 .. 10^8 with rejection draws and with FDR draws."""
    import torch

    import paper_1508_03167_gb300 as ms

    n = (1 << 26) if args.small else N_PERM
    B = TUNED_B["perm"]
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    res = {}
    for tag, flags in (("single_levels", ms.MS_FLAG_GLOBAL_LEVELS | ms.MS_FLAG_SINGLE_LEVELS),
                       ("literal", ms.MS_FLAG_LITERAL), ("fdr", ms.MS_FLAG_FDR),
                       ("literal_fdr", ms.MS_FLAG_LITERAL | ms.MS_FLAG_FDR),
                       ("balanced_word", ms.MS_FLAG_BALANCED)):
        p = ms.params(B=B, fuse_depth=0, flags=flags)
        ws = torch.empty(ms.ms_workspace_bytes(n, 4, p), dtype=torch.uint8, device="cuda")

        def call():
            st = ms.ms_perm(out.data_ptr(), n, SEED, ws.data_ptr(), ws.numel(), p, s.cuda_stream)
            if st != ms.MS_OK:
                raise ms.MsError(st, "ms_perm")

        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            call()
        e1.record(s)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / steps
        res[tag] = {"ms": round(t, 3), "gelem_per_s": round(n / (t * 1e-3) / 1e9, 4)}
        del ws
        torch.cuda.empty_cache()
    del out
    table = []
    for nn in (10**5, 10**6, 10**7, 10**8):
        rej = ms.random_bits(nn, 1, B=1024)
        fdr = ms.random_bits(nn, 1, B=1024, flags=ms.MS_FLAG_FDR)
        table.append({"n": nn, "bits_rejection": rej["total_bits"], "bits_fdr": fdr["total_bits"],
                      "fdr_over_log2_n_factorial": round(
                          fdr["total_bits"] / (math.lgamma(nn + 1) / math.log(2)), 5)})
    return {"config": {"workload": f"perm of n={n} uint32, seed {SEED}, B={B}, fuse_depth 0, "
                                   "every level one global pass", "n": n, "B": B},
            "times": res,
            "random_bits_B1024_seed1": table,
            "note": "Table 1 (paper): Fisher-Yates 1,631,434 / 19,550,941 / 229,329,728 / "
                    "2,628,248,831 and MergeShuffle 1,636,560 / 19,686,051 / 231,641,075 / "
                    "2,650,387,993 bits for n = 1e5 .. 1e8 (its cutoff is not stated)"}


def run_serve(args) -> dict:
    """Poisson arrivals of perm(n) requests, n log-uniform in [2^10, 2^26], own seeds, under a
    40 GB device-memory cap: the offered 20k req/s (about 121 Gelem/s) overloads one GPU, so the
    window is short; a sub-saturation rate is served too, and one-at-a-time is the baseline."""
    import torch

    from paper_1508_03167_gb300 import serve

    import paper_1508_03167_gb300 as ms

    cap = 40 * (1 << 30)
    out = {}
    # one B for every request (results must not depend on which batch a request joins): the
    # autotuner's batch row for the request-size distribution
    B = ms.resolve_batch(
        [r.n for r in serve.make_requests(args.serve_sub_rate, args.serve_sub_window, 10, 26)],
        4, B=args.B_perm, flags=ms.MS_FLAG_PERM).B
    for tag, rate, dur in (("overload_20k_per_s", 20_000, args.serve_window),
                           ("sub_saturation", args.serve_sub_rate, args.serve_sub_window)):
        reqs = serve.make_requests(rate, dur, 10, 26, seed_base=1)
        srv = serve.Server(arena_bytes=cap, B=B, max_inflight=args.serve_inflight)
        st = srv.run(reqs, time_limit=600)
        del srv
        torch.cuda.empty_cache()
        st["offered_rate_per_s"] = rate
        st["window_s"] = dur
        st["limiter"] = ("device memory (the arena held its cap)"
                         if st["arena_peak_bytes"] > 0.9 * cap else
                         f"launch slots (max_inflight = {args.serve_inflight}; the arena peaked "
                         f"at {st['arena_peak_bytes'] / 2**30:.2f} of "
                         f"{cap / 2**30:.0f} GiB)")
        out[tag] = st
    reqs = serve.make_requests(args.serve_sub_rate, args.serve_sub_window, 10, 26, seed_base=1)
    out["one_at_a_time_sub_saturation"] = serve.one_at_a_time(reqs, B=B)
    reqs = serve.make_requests(20_000, args.serve_window, 10, 26, seed_base=1)
    out["one_at_a_time_overload_20k_per_s"] = serve.one_at_a_time(reqs, B=B)
    ov, one = out["overload_20k_per_s"], out["one_at_a_time_overload_20k_per_s"]
    return {
        "metric": "Gelem/s", "value": round(ov["gelem_per_s"], 4),
        "unit": "Gelem/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "dtype": "u32",
        "config": {"workload": "serving: Poisson perm(n) requests, n log-uniform in "
                               "[2^10, 2^26], own seeds, 40 GB device-memory cap, continuous "
                               f"batching over {args.serve_inflight} streams (small requests "
                               "batched, large alone)", "B": B,
                   "window_note": f"{args.serve_window} s of the 20k/s arrivals (the offered "
                                  "load, about 121 Gelem/s, is above what one GPU serves, so "
                                  "the queue and the tail latency grow with the window)"},
        "p50_s": ov["latency_s"]["p50"], "p99_s": ov["latency_s"]["p99"],
        "speedup_vs_one_at_a_time": round(ov["gelem_per_s"] / one["gelem_per_s"], 2),
        "serving": out,
    }


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        print(json.dumps(run_batched(args, large=False)), flush=True)
    elif args.workload == "batched-large":
        print(json.dumps(run_batched(args, large=True)), flush=True)
    elif args.workload == "serve":
        print(json.dumps(run_serve(args)), flush=True)
    elif args.workload == "rs":
        print(json.dumps(run_rs(args)), flush=True)
    elif args.workload == "variants":
        print(json.dumps(run_literal_fdr(args)), flush=True)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
