"""Batched form through the C ABI: every instance of a batch equals its single-call result and
the oracle, bit for bit, whatever else is in the batch (sizes spanning the persistent engine and
the single-instance path for the largest ones); a prepared run replays from a CUDA graph."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1508_03167_gb300 as ms
from paper_1508_03167_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run_batch(tensors, w, base_seed, B, perm, seeds=None):
    import torch

    flags = ms.MS_FLAG_PERM if perm else 0
    p = ms.params(B=B, flags=flags)
    ns = [t.shape[0] for t in tensors]
    ptrs = [t.data_ptr() if t.shape[0] else 0 for t in tensors]
    nbytes = ms.ms_batch_workspace_bytes(ns, w, p)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = ms.ms_shuffle_batch(ptrs, ns, w, seeds, base_seed, ws.data_ptr(), nbytes, p,
                             torch.cuda.current_stream().cuda_stream)
    assert st == ms.MS_OK, ms.ms_status_string(st)
    torch.cuda.synchronize()


@pytest.mark.parametrize("B", [64, 1024])
def test_perm_batch_matches_oracle(B):
    import torch

    sizes = [0, 1, 2, 5, 100, 1000, 4097, 65537, 300017, 1 << 20, (1 << 22) + 3]
    outs = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in sizes]
    _run_batch(outs, 4, 100, B, perm=True)
    for i, (n, o) in enumerate(zip(sizes, outs)):
        want, _ = oracle.perm(n, 100 + i, B)
        assert np.array_equal(o.cpu().numpy().view(np.uint32), want), (i, n)


def test_perm_batch_log_uniform_sizes_match_single_calls():
    import torch

    sizes = [int(x) for x in inputs.batch_sizes_log_uniform(300, 6, 17)]
    B = 128
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    _run_batch(outs, 4, 7, B, perm=True)
    for i in range(len(sizes)):
        single = ms.perm(sizes[i], 7 + i, B=B)
        assert torch.equal(outs[i], single), i
    for i in (0, 1, 50, 299):
        want, _ = oracle.perm(sizes[i], 7 + i, B)
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("w", [8, 16])
def test_shuffle_batch_widths(w):
    import torch

    sizes = [3, 777, 40961, 200003]
    host = []
    for j, n in enumerate(sizes):
        host.append(inputs.records16(n) if w == 16 else inputs.values_u64(n, j))
    devs = [torch.from_numpy(h.view(np.uint8).reshape(h.shape[0], w).copy()).cuda()
            for h in host]
    seeds = [11, 5, 2**40 + 3, 0]
    _run_batch(devs, w, 0, 256, perm=False, seeds=seeds)
    for j, n in enumerate(sizes):
        want, _ = oracle.shuffle(host[j], seeds[j], 256)
        got = devs[j].cpu().numpy().view(host[j].dtype).reshape(host[j].shape)
        assert np.array_equal(got, want), j


def test_prepared_batch_replays_from_a_cuda_graph():
    import torch

    sizes = [5000, 123457, 1 << 18, 70001]
    B = 128
    p = ms.params(B=B, flags=ms.MS_FLAG_PERM)
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
    ptrs = [o.data_ptr() for o in outs]
    nbytes = ms.ms_batch_workspace_bytes(sizes, 4, p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert ms.ms_batch_prepare(ptrs, sizes, 4, None, 3, ws.data_ptr(), nbytes, p,
                                   s.cuda_stream) == ms.MS_OK
        # one eager run first (sets kernel attributes outside the capture)
        assert ms.ms_batch_run(ptrs, sizes, 4, None, 3, ws.data_ptr(), nbytes, p,
                               s.cuda_stream) == ms.MS_OK
    s.synchronize()
    for o in outs:
        o.fill_(-1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert ms.ms_batch_run(ptrs, sizes, 4, None, 3, ws.data_ptr(), nbytes, p,
                               s.cuda_stream) == ms.MS_OK
    for _ in range(2):
        for o in outs:
            o.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        for i, n in enumerate(sizes):
            want, _ = oracle.perm(n, 3 + i, B)
            assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), want), i


def test_autotuned_batch_runs_every_instance_at_the_batch_B():
    """B = 0 in a batch resolves one B from the median size (the tuning table's batch row); every
    instance, the large ones on the single-instance path included, uses it."""
    import torch

    sizes = [100, 3000, 65537, 1 << 20, (1 << 22) + 5]
    B = ms.resolve_batch(sizes, 4, B=0).B
    outs = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for n in sizes]
    _run_batch(outs, 4, 40, 0, perm=True)
    for i, n in enumerate(sizes):
        want, _ = oracle.perm(n, 40 + i, B)
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), want), (i, n)


def test_two_threads_batches_with_several_large_instances():
    """Two host threads each run, on their own stream, batches with several instances above the
    engine's limit (forked onto side streams and joined back). Each thread's side streams belong
    to its own stream, so each batch's large instances start only after that thread's earlier
    work on its stream: every thread first fills its buffers with a marker on its stream, and the
    results must equal the single calls bit for bit on every round."""
    import threading

    import torch

    B = 256
    jobs = {0: [(1 << 22) + 5, (1 << 22) + 1001, 70_001], 1: [(1 << 22) + 77, (1 << 22) + 3, 999]}
    outs, errs = {}, []

    def work(tid, sizes):
        try:
            s = torch.cuda.Stream()
            p = ms.params(B=B, flags=ms.MS_FLAG_PERM)
            ptrs_t = [torch.empty(n, dtype=torch.int32, device="cuda") for n in sizes]
            nbytes = ms.ms_batch_workspace_bytes(sizes, 4, p)
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            ptrs = [t.data_ptr() for t in ptrs_t]
            for rnd in range(3):
                with torch.cuda.stream(s):
                    for t in ptrs_t:
                        t.fill_(-1 - rnd)
                assert ms.ms_shuffle_batch(ptrs, sizes, 4, None, 40 + 10 * tid, ws.data_ptr(),
                                           nbytes, p, s.cuda_stream) == ms.MS_OK
            s.synchronize()
            outs[tid] = [t.clone() for t in ptrs_t]
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=work, args=(i, j)) for i, j in jobs.items()]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for tid, sizes in jobs.items():
        for i, n in enumerate(sizes):
            assert torch.equal(outs[tid][i], ms.perm(n, 40 + 10 * tid + i, B=B)), (tid, i)
