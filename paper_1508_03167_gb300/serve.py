"""Serving loop for MergeShuffle requests: continuous batching under a device-memory cap.

Requests (n, seed) arrive over time. The server keeps every buffer in one fixed device arena
(allocated once), admits a pending request only when its memory fits the arena, and keeps up to
`max_inflight` launches on the GPU at once, one CUDA stream each: requests that arrive while
others run are admitted as soon as memory and a launch slot free up, and their kernels overlap
with the work already in flight. Small requests (n <= small_cap) go out together as one call of
the batched form (persistent CTA-per-instance engine); each larger request goes out alone, so it
never waits for a batch and no small request waits for it. Completion times come from CUDA events on the batch's stream, so latency = completion on
the GPU timeline - arrival, both measured from the same start.

The arena allocator and the admission bookkeeping are plain Python (testable without a GPU);
all shuffling happens in the CUDA library.
"""
from __future__ import annotations

import bisect
import dataclasses
import time

ALIGN = 256


class Arena:
    """First-fit allocator over [0, capacity) with coalescing frees; offsets are ALIGN-aligned."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.free = [(0, capacity)]  # sorted (offset, size)
        self.used = 0
        self.peak = 0

    @staticmethod
    def _round(n: int) -> int:
        return (n + ALIGN - 1) // ALIGN * ALIGN

    def alloc(self, nbytes: int):
        size = self._round(max(nbytes, 1))
        for i, (off, sz) in enumerate(self.free):
            if sz >= size:
                if sz == size:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + size, sz - size)
                self.used += size
                self.peak = max(self.peak, self.used)
                return off, size
        return None

    def release(self, block) -> None:
        off, size = block
        self.used -= size
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, size))
        # coalesce with the neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            o, s = self.free[i]
            self.free[i] = (o, s + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            o, s = self.free[i - 1]
            self.free[i - 1] = (o, s + self.free[i][1])
            self.free.pop(i)


@dataclasses.dataclass
class Request:
    rid: int
    n: int
    seed: int
    arrival: float           # seconds from the start
    admitted: float = -1.0
    done: float = -1.0
    out: tuple | None = None  # arena block of the result


def percentiles(xs, ps=(50, 99)):
    import numpy as np

    if len(xs) == 0:
        return {f"p{p}": None for p in ps}
    a = np.asarray(xs)
    return {f"p{p}": float(np.percentile(a, p)) for p in ps}


class Server:
    """Continuous-batching server over the batched C entry points."""

    def __init__(self, arena_bytes: int, B: int = 128, max_inflight: int = 4,
                 max_batch: int = 4096, device=None, keep_results: bool = False,
                 small_cap: int = 1 << 18):
        import torch

        import paper_1508_03167_gb300 as ms

        if B < 1:
            # B = 0 would resolve per batch (by its median size), so a request's result would
            # depend on which requests it was batched with; resolve one B up front instead
            raise ValueError("the server needs an explicit cutoff B (see ms.resolve_batch)")
        self.ms = ms
        self.torch = torch
        self.B = B
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.keep_results = keep_results
        self.small_cap = small_cap
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.arena_bytes = arena_bytes
        self.mem = torch.empty(arena_bytes, dtype=torch.uint8, device=self.device)
        self.base = self.mem.data_ptr()
        self.arena = Arena(arena_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max_inflight)]
        self.params = ms.params(B=B, flags=ms.MS_FLAG_PERM)
        self.results = {}

    # -- memory a batch needs: its workspace (engine ping-pong buffers, scratch, table, one
    #    single-instance workspace for large requests) plus each request's output buffer
    FIXED_WS = 96 << 20          # per-batch scratch and table (upper estimate)
    ENGINE_MAX_N = 1 << 22       # larger requests run the single-instance path in a batch

    def _batch_ws_bytes(self, ns):
        return self.ms.ms_batch_workspace_bytes(ns, 4, self.params)

    def _large_ws(self, n):
        return self.ms.ms_workspace_bytes(n, 4, self.ms.params(B=self.B))

    def _footprint(self, n):
        """Arena bytes a request needs when admitted alone: its output, the batch workspace of
        a one-request batch and the fixed per-batch estimate the admission test adds."""
        extra = 4 * n if n <= self.ENGINE_MAX_N else self._large_ws(n)
        ws = self.ms.ms_batch_workspace_bytes([n], 4, self.params)
        return max(self.FIXED_WS + extra + 4 * n, Arena._round(4 * n) + Arena._round(ws))

    def _admit(self, group):
        """Allocate outputs for a prefix of `group` and the batch workspace; returns the admitted
        requests (possibly none). The workspace block is left in self._ws_blk."""
        batch, ns = [], []
        est = self.FIXED_WS
        for r in group:
            extra = 4 * r.n if r.n <= self.ENGINE_MAX_N else self._large_ws(r.n)
            if self.arena.capacity - self.arena.used < est + extra + 4 * r.n:
                break
            out_blk = self.arena.alloc(4 * r.n)
            if out_blk is None:
                break
            r.out = out_blk
            batch.append(r)
            ns.append(r.n)
            est += extra
        self._ws_blk = None
        while batch:
            self._ws_blk = self.arena.alloc(self._batch_ws_bytes(ns))
            if self._ws_blk is not None:
                break
            r = batch.pop()
            ns.pop()
            self.arena.release(r.out)
            r.out = None
        return batch

    def run(self, requests, time_limit: float = 600.0) -> dict:
        """Serve `requests` (sorted by arrival). Returns latency/throughput statistics."""
        torch, ms = self.torch, self.ms
        pending = []            # arrived, not admitted (FIFO)
        inflight = []           # (event, stream index, requests, ws block)
        free_streams = list(range(self.max_inflight))
        nxt = 0
        done = []
        rejected = []
        timed_out = False
        start_evt = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        start_evt.record(self.streams[0])
        elems = 0
        while True:
            now = time.perf_counter() - t0
            while nxt < len(requests) and requests[nxt].arrival <= now:
                r = requests[nxt]
                nxt += 1
                # a request that would not fit even in an empty arena can never be admitted:
                # reject it on arrival rather than leave it pending for ever
                if self._footprint(r.n) > self.arena.capacity:
                    rejected.append(r)
                else:
                    pending.append(r)
            # completions (host polls the batch events; the GPU timestamp is the completion)
            still = []
            for evt, si, reqs, wsb in inflight:
                if evt.query():
                    t_done = start_evt.elapsed_time(evt) * 1e-3
                    if self.keep_results:
                        # copy the results out on the batch's own stream and wait for the copy:
                        # the arena blocks are reused by later batches on other streams
                        with torch.cuda.stream(self.streams[si]):
                            for r in reqs:
                                off = r.out[0]
                                self.results[r.rid] = self.mem[off:off + 4 * r.n].view(
                                    torch.int32).clone()
                        self.streams[si].synchronize()
                    for r in reqs:
                        r.done = t_done
                        self.arena.release(r.out)
                        done.append(r)
                        elems += r.n
                    self.arena.release(wsb)
                    free_streams.append(si)
                else:
                    still.append((evt, si, reqs, wsb))
            inflight = still
            # admission: small requests (n <= small_cap) go out together as one batch on a free
            # stream; every larger request goes out alone on its own free stream. Requests are
            # taken in arrival order as long as their buffers fit the arena.
            if free_streams and pending:
                smalls = [r for r in pending if r.n <= self.small_cap]
                groups = []
                if smalls:
                    groups.append(smalls[:self.max_batch])
                groups += [[r] for r in pending if r.n > self.small_cap]
                launched = set()
                for group in groups:
                    if not free_streams:
                        break
                    batch = self._admit(group)
                    if not batch:
                        continue
                    ns = [r.n for r in batch]
                    ws_blk = self._ws_blk
                    si = free_streams.pop()
                    st = self.streams[si]
                    ptrs = [self.base + r.out[0] for r in batch]
                    seeds = [r.seed for r in batch]
                    for r in batch:
                        r.admitted = now
                        launched.add(r.rid)
                    rc = ms.ms_shuffle_batch(ptrs, ns, 4, seeds, 0, self.base + ws_blk[0],
                                             ws_blk[1], self.params, st.cuda_stream)
                    if rc != ms.MS_OK:
                        raise ms.MsError(rc, "ms_shuffle_batch")
                    evt = torch.cuda.Event(enable_timing=True)
                    evt.record(st)
                    inflight.append((evt, si, batch, ws_blk))
                if launched:
                    pending = [r for r in pending if r.rid not in launched]
            if nxt >= len(requests) and not pending and not inflight:
                break
            if time.perf_counter() - t0 > time_limit:
                timed_out = True
                break
            if not (free_streams and pending):
                time.sleep(20e-6)
        torch.cuda.synchronize(self.device)
        wall = time.perf_counter() - t0
        lat = [r.done - r.arrival for r in done]
        last = max((r.done for r in done), default=0.0)
        first = min((r.arrival for r in requests), default=0.0)
        stats = {
            "requests": len(requests),
            "completed": len(done),
            "elements": elems,
            "gelem_per_s": elems / max(last - first, 1e-9) / 1e9,
            "latency_s": {**percentiles(lat), "max": max(lat) if lat else None,
                          "mean": sum(lat) / len(lat) if lat else None},
            "arena_peak_bytes": self.arena.peak,
            "arena_bytes": self.arena_bytes,
            "wall_s": wall,
            "rejected": len(rejected),
            "time_limit_hit": timed_out,
            # requests still waiting (never admitted) or not yet arrived when the run ended;
            # the latency percentiles cover completed requests only
            "pending_at_end": len(pending) + (len(requests) - nxt),
            "inflight_at_end": sum(len(reqs) for _, _, reqs, _ in inflight),
        }
        return stats


def one_at_a_time(requests, B: int = 128, device=None) -> dict:
    """Baseline: the same arrivals served strictly one request at a time with ms_perm."""
    import torch

    import paper_1508_03167_gb300 as ms

    dev = device or torch.device("cuda", torch.cuda.current_device())
    p = ms.params(B=B)
    nmax = max(r.n for r in requests)
    out = torch.empty(nmax, dtype=torch.int32, device=dev)
    ws = torch.empty(ms.ms_workspace_bytes(nmax, 4, p), dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    start_evt = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    start_evt.record(s)
    lat = []
    elems = 0
    last = 0.0
    for r in requests:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        rc = ms.ms_perm(out.data_ptr(), r.n, r.seed, ws.data_ptr(), ws.numel(), p, s.cuda_stream)
        if rc != ms.MS_OK:
            raise ms.MsError(rc, "ms_perm")
        e = torch.cuda.Event(enable_timing=True)
        e.record(s)
        e.synchronize()
        done = start_evt.elapsed_time(e) * 1e-3
        lat.append(done - r.arrival)
        elems += r.n
        last = done
    first = min(r.arrival for r in requests)
    return {"requests": len(requests), "elements": elems,
            "gelem_per_s": elems / max(last - first, 1e-9) / 1e9,
            "latency_s": {**percentiles(lat), "max": max(lat), "mean": sum(lat) / len(lat)}}


def make_requests(rate_hz: float, duration_s: float, lo_log2: float, hi_log2: float,
                  seed_base: int = 1, max_requests: int | None = None):
    """Poisson arrivals at rate_hz for duration_s; n log-uniform in [2^lo, 2^hi]."""
    from . import inputs

    t = inputs.poisson_arrivals(rate_hz, duration_s)
    if max_requests is not None:
        t = t[:max_requests]
    sizes = inputs.batch_sizes_log_uniform(len(t), lo_log2, hi_log2, stream=inputs.S_SIZE + 7)
    return [Request(rid=i, n=int(n), seed=seed_base + i, arrival=float(a))
            for i, (a, n) in enumerate(zip(t, sizes))]
