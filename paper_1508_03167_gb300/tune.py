"""Autotuner: picks the cutoff B, the fusion depth and the merge-level mode per element width and
size bucket by timing the CUDA library on the GPU, and writes the table the library's B = 0
lookup uses (``csrc/ms_tune_table.h``, built in) plus a JSON copy that can be installed at run
time with ``ms_tune_install``.

The paper leaves the cutoff open: its driver (Algorithm 2) only needs 2^c nearly equal blocks,
and the appendix listing takes the cutoff as a parameter. B is part of the result's definition,
so the tuner only changes which B a call with B = 0 resolves to; every tuned choice is recorded
in the table. The fusion depth and the level mode never change the result. A row's B is a block
size: the library runs a call of n elements with the cutoff whose blocks are nearest to it
(``row_cutoff``), and the tuner times each candidate the same way.

Usage on a GPU:  python -m paper_1508_03167_gb300.tune [--quick] [--header] [--json PATH]
Built-in table from a saved JSON table:  python -m paper_1508_03167_gb300.tune --from-json PATH
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "ms_tune_table.h")
JSON_PATH = os.path.join(HERE, "tune_table.json")

B_CANDIDATES = (32, 64, 128, 256, 512, 1024)
# (fuse_depth, flags) alternatives per B: the planner's fusion depth, none, or 3 .. 6 levels in
# the tile kernel; the default small levels or per-CTA ones; one data pass per global level or
# fused pairs of them
MODE_CANDIDATES = ((-1, 0), (0, 0), (0, 0x8), (0, 0x80), (0, 0x100), (3, 0), (4, 0), (5, 0),
                   (6, 0), (5, 0x80), (5, 0x100))
# size points per width: log2 n (the largest fits a 2 x n x w footprint comfortably); sizes are
# 2^k for w = 4 and 2^k + 17 otherwise (uneven halves), except that the last 16-byte point is
# the 300,000,017-record workload itself
SINGLE_POINTS = {4: (10, 14, 18, 22, 26, 30), 8: (10, 14, 18, 22, 26, 29),
                 16: (10, 14, 18, 22, 26, 29)}
EXACT_N = {(16, 29): 300_000_017}
QUICK_POINTS = {4: (14, 22, 26), 8: (22,), 16: (22,)}


def pick(timings: dict) -> tuple:
    """The fastest candidate of {candidate: [milliseconds...]} by median; ties go to the first
    candidate in insertion order."""
    best, best_t = None, None
    for cand, ts in timings.items():
        t = statistics.median(ts)
        if best_t is None or t < best_t:
            best, best_t = cand, t
    return best


def buckets(points) -> list[int]:
    """log2n_max of each size point: a point covers sizes up to halfway to the next one; the
    last covers everything above."""
    pts = sorted(points)
    out = []
    for i, p in enumerate(pts):
        out.append((p + pts[i + 1]) // 2 if i + 1 < len(pts) else 64)
    return out


def header_text(rows) -> str:
    lines = [
        "// Built-in autotuner table: {w, batch, log2n_max, B, fuse_depth, flags}, one row per",
        "// element width, call form and size bucket. Written by paper_1508_03167_gb300/tune.py",
        "// from timings on a GB300 (median of timed calls per candidate).",
    ]
    for r in rows:
        lines.append(f"{{{r['w']}, {r['batch']}, {r['log2n_max']}, {r['B']}, "
                     f"{r['fuse_depth']}, {r['flags']}}},")
    return "\n".join(lines) + "\n"


def parse_header(text: str) -> list[dict]:
    rows = []
    for line in text.splitlines():
        line = line.strip()
        if not line.startswith("{"):
            continue
        vals = [int(v) for v in line.strip("{},").split(",")]
        rows.append(dict(zip(("w", "batch", "log2n_max", "B", "fuse_depth", "flags"), vals)))
    return rows


def row_cutoff(n: int, w: int, B: int) -> int:
    """The cutoff a single call of n elements of width w runs with when the table's row holds
    block size B: the library's own rule, read through a one-row table (host only)."""
    from . import ms_tune_install, resolve

    ms_tune_install([dict(w=w, batch=0, log2n_max=64, B=B, fuse_depth=-1, flags=0)])
    try:
        return resolve(n, w, B=0).B
    finally:
        ms_tune_install([])  # back to the built-in table


# ------------------------------------------------------------------ GPU timing ----------------
def _time(fn, reps: int, warmup: int = 2) -> list[float]:
    import torch

    for _ in range(warmup):
        fn()
    out = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def time_single(n: int, w: int, B: int, fuse_depth: int, flags: int, reps: int) -> list[float]:
    import torch

    from . import MS_OK, MsError, ms_perm, ms_shuffle, ms_workspace_bytes, params

    p = params(B=B, fuse_depth=fuse_depth, flags=flags)
    ws = torch.empty(ms_workspace_bytes(n, w, p), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    if w == 4:
        x = torch.empty(n, dtype=torch.int32, device="cuda")

        def fn():
            st = ms_perm(x.data_ptr(), n, 7, ws.data_ptr(), ws.numel(), p, s)
            if st != MS_OK:
                raise MsError(st, "ms_perm")
    else:
        x = torch.zeros((n, w // 4), dtype=torch.int32, device="cuda")

        def fn():
            st = ms_shuffle(x.data_ptr(), n, w, 7, ws.data_ptr(), ws.numel(), p, s)
            if st != MS_OK:
                raise MsError(st, "ms_shuffle")
    try:
        return _time(fn, reps)
    finally:
        del x, ws
        torch.cuda.empty_cache()


def batch_sizes(w: int) -> list[int]:
    """The batched workload each width is tuned on: 4096 sizes log-uniform in [2^6, 2^20] for
    permutations (w = 4), 1024 for the wider records."""
    from . import inputs

    k = 4096 if w == 4 else 1024
    return [int(v) for v in inputs.batch_sizes_log_uniform(k, 6.0, 20.0)]


def time_batch(ns, w: int, B: int, fuse_depth: int, flags: int, reps: int) -> list[float]:
    import torch

    from . import (MS_FLAG_PERM, MS_OK, MsError, ms_batch_prepare, ms_batch_run,
                   ms_batch_workspace_bytes, params)

    fl = flags | (MS_FLAG_PERM if w == 4 else 0)
    p = params(B=B, fuse_depth=fuse_depth, flags=fl)
    total = sum(ns)
    store = torch.zeros(total * (w // 4), dtype=torch.int32, device="cuda")
    ptrs, off = [], 0
    for n in ns:
        ptrs.append(store.data_ptr() + off * w)
        off += n
    ws = torch.empty(ms_batch_workspace_bytes(ns, w, p), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    st = ms_batch_prepare(ptrs, ns, w, None, 1, ws.data_ptr(), ws.numel(), p, s)
    if st != MS_OK:
        raise MsError(st, "ms_batch_prepare")

    def fn():
        st = ms_batch_run(ptrs, ns, w, None, 1, ws.data_ptr(), ws.numel(), p, s)
        if st != MS_OK:
            raise MsError(st, "ms_batch_run")
    try:
        return _time(fn, reps)
    finally:
        del store, ws
        torch.cuda.empty_cache()


def tune(quick: bool = False, reps: int = 5, log=print) -> list[dict]:
    rows = []
    points = QUICK_POINTS if quick else SINGLE_POINTS
    for w, pts in points.items():
        for lg, lmax in zip(sorted(pts), buckets(pts)):
            n = EXACT_N.get((w, lg), (1 << lg) + (0 if w == 4 else 17))
            timings = {}
            for B in B_CANDIDATES:
                if B >= n:
                    continue
                for fd, fl in MODE_CANDIDATES:
                    if fl in (0x80, 0x100) and lg < 20:
                        continue  # few global levels: nothing to fuse
                    timings[(B, fd, fl)] = time_single(n, w, row_cutoff(n, w, B), fd, fl,
                                                       reps)
            B, fd, fl = pick(timings)
            log(f"single w={w:2d} n=2^{lg}: B={B} fuse_depth={fd} flags={fl:#x} "
                f"({statistics.median(timings[(B, fd, fl)]):.3f} ms)")
            rows.append(dict(w=w, batch=0, log2n_max=lmax, B=B, fuse_depth=fd, flags=fl))
        ns = batch_sizes(w)
        timings = {}
        for B in B_CANDIDATES:
            timings[(B, -1, 0)] = time_batch(ns, w, B, -1, 0, reps)
        B, fd, fl = pick(timings)
        log(f"batch  w={w:2d} k={len(ns)}: B={B} ({statistics.median(timings[(B, fd, fl)]):.3f} ms)")
        rows.append(dict(w=w, batch=1, log2n_max=64, B=B, fuse_depth=fd, flags=fl))
    return rows


def save_json(rows, path: str = JSON_PATH) -> None:
    with open(path, "w") as f:
        json.dump(rows, f, indent=1)


def load_json(path: str = JSON_PATH) -> list[dict]:
    with open(path) as f:
        return json.load(f)


def install(rows) -> None:
    from . import ms_tune_install

    ms_tune_install(rows)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--quick", action="store_true", help="few size points (a smoke run)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--json", default=JSON_PATH, help="where to write the JSON table")
    ap.add_argument("--header", action="store_true",
                    help="also rewrite the built-in table csrc/ms_tune_table.h")
    ap.add_argument("--from-json", default=None,
                    help="no timing: rewrite the built-in table from this JSON table")
    a = ap.parse_args(argv)
    if a.from_json:
        with open(HEADER, "w") as f:
            f.write(header_text(load_json(a.from_json)))
        return 0
    rows = tune(quick=a.quick, reps=a.reps)
    save_json(rows, a.json)
    if a.header:
        with open(HEADER, "w") as f:
            f.write(header_text(rows))
    print(json.dumps(rows))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
