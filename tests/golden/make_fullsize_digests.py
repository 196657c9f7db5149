"""Writes fullsize_digests.txt: SHA-256 digests of the CPU oracle's outputs on the workloads the
benchmark times, at the cutoff B each of them resolves to.

This script is the only writer of those values. It calls the oracle (``oracle/``) and the seeded
input generators (``paper_1508_03167_gb300/inputs.py``, loaded by path so that nothing else of the
package runs); it never loads the CUDA library. The result definition it pins is Algorithm 2 of
the paper (Fisher-Yates on the base blocks of the appendix listing's block split, then the merge
levels of Algorithm 3), on the stream definition MS-Philox v1.

Workloads (B is what the built-in tuning table resolves each one to; the GPU test checks that the
table still resolves them so, so the digests stay tied to what the benchmark runs):
  c1_perm        perm(2^20), seed 1, B = 1024 (the small configuration; B fixed by it)
  c2a_perm       perm(2^30), seed 7, B = 512
  c2b_records    shuffle of 300,000,017 16-byte records {u32 key = i, 12-byte splitmix64 payload},
                 seed 7, B = 572
  c3_batch       the 4096 perm(n_i) of the batched workload (n_i log-uniform in [2^6, 2^20],
                 seed_i = 1 + i), B = 256: one digest over the instances' outputs in order
  c4_u64_<i>     instance i of the batched-large workload (uint64 splitmix64 values, n_i uniform
                 in [10^6, 10^8]), seed 1 + i, B = 256: the largest instance and a small one
  rs_perm        the splitting process (Rao-Sandelius, Fisher-Yates cutoff B) on 2^30 positions,
                 seed 7, B = 512: the comparison workload's perm
  max_perm       perm(2^32 - 1), seed 3, B = 511: the largest n the boundary takes (positions
                 near 2^32 exercise every 32-bit index of the GPU path)
  rs_max         the splitting process on 2^32 - 1 positions, seed 5, B = 512

Run:  python tests/golden/make_fullsize_digests.py [name ...]   (all rows: about an hour on one
core, ~38 GB RAM; with names, only those rows are recomputed and the others kept)
"""
from __future__ import annotations

import hashlib
import importlib.util
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize_digests.txt")
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402


def _inputs():
    spec = importlib.util.spec_from_file_location(
        "ms_inputs", os.path.join(ROOT, "paper_1508_03167_gb300", "inputs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


inputs = _inputs()

C1 = dict(name="c1_perm", n=1 << 20, w=4, seed=1, B=1024)
C2A = dict(name="c2a_perm", n=1 << 30, w=4, seed=7, B=512)
C2B = dict(name="c2b_records", n=300_000_017, w=16, seed=7, B=572)
C3_B = 256
C4_B = 256
RS = dict(name="rs_perm", n=1 << 30, w=4, seed=7, B=512)
MAX = dict(name="max_perm", n=(1 << 32) - 1, w=4, seed=3, B=511)
RS_MAX = dict(name="rs_max", n=(1 << 32) - 1, w=4, seed=5, B=512)


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main(only: set[str]) -> None:
    rows = {}
    if only and os.path.exists(OUT):
        with open(OUT) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    rows[line.split()[0]] = line.strip()

    def want(name):
        return not only or name in only or (name.startswith("c4_u64_") and "c4" in only)

    def emit(name, n, w, seed, B, digest, dt):
        rows[name] = f"{name} {n} {w} {seed} {B} {digest}"
        print(f"{name}: n={n} w={w} seed={seed} B={B} {digest} ({dt:.1f} s)", flush=True)

    for cfg in (C1, C2A, MAX):
        if not want(cfg["name"]):
            continue
        t = time.time()
        out, _ = oracle.perm(cfg["n"], cfg["seed"], cfg["B"])
        emit(cfg["name"], cfg["n"], 4, cfg["seed"], cfg["B"], sha(out), time.time() - t)
        del out

    if want(C2B["name"]):
        t = time.time()
        rec = inputs.records16(C2B["n"])
        out, _ = oracle.shuffle(rec, C2B["seed"], C2B["B"])
        del rec
        emit(C2B["name"], C2B["n"], 16, C2B["seed"], C2B["B"], sha(out), time.time() - t)
        del out

    # batched: every instance's permutation, concatenated in instance order
    if want("c3_batch"):
        t = time.time()
        sizes = [int(x) for x in inputs.batch_sizes_log_uniform(4096, 6, 20)]
        h = hashlib.sha256()
        for i, n in enumerate(sizes):
            out, _ = oracle.perm(n, 1 + i, C3_B)
            h.update(out.tobytes())
        emit("c3_batch", sum(sizes), 4, 1, C3_B, h.hexdigest(), time.time() - t)

    # batched large: the largest instance, and the smallest (which the batch engine takes)
    big = [int(x) for x in inputs.batch_sizes_uniform(64, 10**6, 10**8)]
    for i in (max(range(64), key=lambda j: big[j]), min(range(64), key=lambda j: big[j])):
        if not want(f"c4_u64_{i}"):
            continue
        t = time.time()
        vals = inputs.values_u64(big[i], i)
        out, _ = oracle.shuffle(vals, 1 + i, C4_B)
        del vals
        emit(f"c4_u64_{i}", big[i], 8, 1 + i, C4_B, sha(out), time.time() - t)
        del out

    for cfg in (RS, RS_MAX):
        if not want(cfg["name"]):
            continue
        t = time.time()
        out, _ = oracle.rs_perm(cfg["n"], cfg["seed"], cfg["B"])
        emit(cfg["name"], cfg["n"], 4, cfg["seed"], cfg["B"], sha(out), time.time() - t)
        del out

    with open(OUT, "w") as f:
        f.write("# SHA-256 of the CPU oracle's output (little-endian element bytes), written by\n"
                "# make_fullsize_digests.py from the oracle alone. Columns: name n w seed B digest.\n"
                "# c3_batch: n is the total of the 4096 instances, seed the first instance's\n"
                "# (instance i takes seed 1 + i); the digest covers the outputs in instance order.\n")
        for r in rows.values():
            f.write(r + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main(set(sys.argv[1:]))
