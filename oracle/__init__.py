"""CPU oracle for MergeShuffle (arXiv 1508.03167) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It wraps the plain single-threaded C restatement in ``ms_oracle.c`` (Algorithms 1-3
of the paper, the appendix listing's block split, and the MS-Philox v1 stream definition) through
ctypes. It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_HDR = os.path.join(_HERE, "ms_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libms_oracle.so")

STABLE = 0
LITERAL = 1
PHILOX = 0
SEQFDR = 2
FDR = 4
BALANCED = 8

# planted mistakes (exhaustive-walk tests only)
PLANT_FY_RANGE = 16
PLANT_TAIL_RANGE = 32
PLANT_NO_TAIL = 64

TAG_COIN = 1
TAG_TAIL = 2
TAG_LEAF = 3
TAG_RS_COIN = 4
TAG_RS_LEAF = 5

_lock = threading.Lock()
_lib = None


class Stats(ctypes.Structure):
    """Random-bit accounting of one run (the random-bit model of Section 1)."""

    _fields_ = [
        ("coin_bits", ctypes.c_uint64),
        ("leaf_bits", ctypes.c_uint64),
        ("tail_bits", ctypes.c_uint64),
        ("leaf_draws", ctypes.c_uint64),
        ("tail_draws", ctypes.c_uint64),
        ("merges", ctypes.c_uint64),
        ("leftover", ctypes.c_uint64),
        ("levels", ctypes.c_uint64),
    ]

    @property
    def total_bits(self) -> int:
        return int(self.coin_bits + self.leaf_bits + self.tail_bits)

    def as_dict(self) -> dict:
        d = {name: int(getattr(self, name)) for name, _ in self._fields_}
        d["total_bits"] = self.total_bits
        return d


def build(force: bool = False) -> str:
    """Compile ms_oracle.c into a shared library with the host C compiler (gcc)."""
    with _lock:
        os.makedirs(_BUILD_DIR, exist_ok=True)
        stale = (
            force
            or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        )
        if stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    vp = ctypes.c_void_p
    p64 = ctypes.POINTER(ctypes.c_uint64)
    lib.ms_oracle_philox.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.ms_oracle_philox.restype = None
    lib.ms_oracle_coin.argtypes = [u64, u32, u32, u64]
    lib.ms_oracle_coin.restype = i32
    lib.ms_oracle_draw.argtypes = [u64, u32, u32, u32, u64, u64, p64]
    lib.ms_oracle_draw.restype = u64
    lib.ms_oracle_draw_fdr.argtypes = [u64, u32, u32, u32, u64, u64, p64]
    lib.ms_oracle_draw_fdr.restype = u64
    lib.ms_oracle_levels.argtypes = [u64, u32]
    lib.ms_oracle_levels.restype = u32
    lib.ms_oracle_shuffle.argtypes = [vp, u64, u32, u64, u32, i32, ctypes.POINTER(Stats)]
    lib.ms_oracle_shuffle.restype = i32
    lib.ms_oracle_perm.argtypes = [vp, u64, u64, u32, i32, ctypes.POINTER(Stats)]
    lib.ms_oracle_perm.restype = i32
    lib.ms_oracle_merge.argtypes = [vp, u64, u64, u64, u32, u32, i32, p64, ctypes.POINTER(Stats)]
    lib.ms_oracle_merge.restype = i32
    lib.ms_oracle_enumerate.argtypes = [u32, u32, i32, vp, vp, p64]
    lib.ms_oracle_enumerate.restype = i32
    lib.ms_oracle_enumerate_merge.argtypes = [u32, u32, i32, vp, vp, p64]
    lib.ms_oracle_enumerate_merge.restype = i32
    lib.ms_oracle_rs_shuffle.argtypes = [vp, u64, u32, u64, u32, i32, ctypes.POINTER(Stats)]
    lib.ms_oracle_rs_shuffle.restype = i32
    lib.ms_oracle_rs_perm.argtypes = [vp, u64, u64, u32, i32, ctypes.POINTER(Stats)]
    lib.ms_oracle_rs_perm.restype = i32
    lib.ms_oracle_enumerate_rs.argtypes = [u32, u32, u32, i32, vp, vp, p64, vp]
    lib.ms_oracle_enumerate_rs.restype = i32
    _lib = lib
    return lib


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.ms_oracle_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def coin(seed: int, level: int, merge_id: int, t: int) -> int:
    return int(_load().ms_oracle_coin(seed, level, merge_id, t))


def draw(seed: int, tag: int, level: int, stream_id: int, pos: int, R: int) -> tuple[int, int]:
    """(value, bits) of the uniform draw in [0, R) of stream (tag, level, id, pos)."""
    bits = ctypes.c_uint64(0)
    v = _load().ms_oracle_draw(seed, tag, level, stream_id, pos, R, ctypes.byref(bits))
    return int(v), int(bits.value)


def draw_fdr(seed: int, tag: int, level: int, stream_id: int, pos: int, R: int
             ) -> tuple[int, int]:
    """(value, bits) of the Fast Dice Roller draw in [0, R) on stream (tag, level, id, pos)."""
    bits = ctypes.c_uint64(0)
    v = _load().ms_oracle_draw_fdr(seed, tag, level, stream_id, pos, R, ctypes.byref(bits))
    return int(v), int(bits.value)


def levels(n: int, B: int) -> int:
    return int(_load().ms_oracle_levels(n, B))


def shuffle(data: np.ndarray, seed: int, B: int, mode: int = STABLE) -> tuple[np.ndarray, Stats]:
    """Return a shuffled copy of a C-contiguous array whose first axis holds the n elements."""
    arr = np.ascontiguousarray(data).copy()
    n = arr.shape[0]
    w = arr.nbytes // n if n else 1
    st = Stats()
    rc = _load().ms_oracle_shuffle(arr.ctypes.data, n, w, seed, B, mode, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_shuffle failed with code {rc}")
    return arr, st


def perm(n: int, seed: int, B: int, mode: int = STABLE) -> tuple[np.ndarray, Stats]:
    out = np.empty(n, dtype=np.uint32)
    st = Stats()
    rc = _load().ms_oracle_perm(out.ctypes.data, n, seed, B, mode, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_perm failed with code {rc}")
    return out, st


def merge(values: np.ndarray, n1: int, seed: int, level: int = 0, merge_id: int = 0,
          mode: int = STABLE) -> tuple[np.ndarray, int, Stats]:
    """One Merge of values[:n1] and values[n1:] (uint32). Returns (output, T, stats)."""
    arr = np.ascontiguousarray(values, dtype=np.uint32).copy()
    n2 = arr.shape[0] - n1
    T = ctypes.c_uint64(0)
    st = Stats()
    rc = _load().ms_oracle_merge(arr.ctypes.data, n1, n2, seed, level, merge_id, mode,
                                 ctypes.byref(T), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_merge failed with code {rc}")
    return arr, int(T.value), st


def _u128(hi_lo: np.ndarray) -> list[int]:
    return [(int(hi_lo[2 * i]) << 64) | int(hi_lo[2 * i + 1]) for i in range(len(hi_lo) // 2)]


def enumerate_perm(n: int, B: int, mode: int = STABLE) -> tuple[list[int], int, int]:
    """Exact output distribution of MergeShuffle on the identity of size n <= 8.

    Returns (numerators indexed by Lehmer rank, common denominator, number of tree leaves)."""
    import math

    nf = math.factorial(n)
    num = np.zeros(2 * nf, dtype=np.uint64)
    den = np.zeros(2, dtype=np.uint64)
    paths = ctypes.c_uint64(0)
    rc = _load().ms_oracle_enumerate(n, B, mode, num.ctypes.data, den.ctypes.data,
                                     ctypes.byref(paths))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_enumerate failed with code {rc}")
    return _u128(num), _u128(den)[0], int(paths.value)


def enumerate_merge(a: int, b: int, mode: int = STABLE) -> tuple[list[int], int, int]:
    """Exact distribution of the first-half position set of one Merge (a + b <= 10)."""
    nm = 1 << (a + b)
    num = np.zeros(2 * nm, dtype=np.uint64)
    den = np.zeros(2, dtype=np.uint64)
    paths = ctypes.c_uint64(0)
    rc = _load().ms_oracle_enumerate_merge(a, b, mode, num.ctypes.data, den.ctypes.data,
                                           ctypes.byref(paths))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_enumerate_merge failed with code {rc}")
    return _u128(num), _u128(den)[0], int(paths.value)


# ------------------------------------------------------------------ splitting process --------
def rs_shuffle(data: np.ndarray, seed: int, B: int, mode: int = PHILOX) -> tuple[np.ndarray, Stats]:
    """Rao-Sandelius splitting process with Fisher-Yates cutoff B on a copy of `data` (first axis
    = the n elements). Stats: coin_bits (bits of the splits), merges (number of splits), levels
    (split levels), leaf_bits / leaf_draws (Fisher-Yates)."""
    arr = np.ascontiguousarray(data).copy()
    n = arr.shape[0]
    w = arr.nbytes // n if n else 1
    st = Stats()
    rc = _load().ms_oracle_rs_shuffle(arr.ctypes.data, n, w, seed, B, mode, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_rs_shuffle failed with code {rc}")
    return arr, st


def rs_perm(n: int, seed: int, B: int, mode: int = PHILOX) -> tuple[np.ndarray, Stats]:
    out = np.empty(n, dtype=np.uint32)
    st = Stats()
    rc = _load().ms_oracle_rs_perm(out.ctypes.data, n, seed, B, mode, ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"ms_oracle_rs_perm failed with code {rc}")
    return out, st


def enumerate_rs(n: int, B: int, max_levels: int, mode: int = 0
                 ) -> tuple[list[int], int, int, int]:
    """Exact walk of the splitting process on the identity of size n <= 6, cut at max_levels
    split levels. Returns (numerators by Lehmer rank over paths that finish, denominator, leaves,
    numerator of the cut-off paths)."""
    import math

    nf = math.factorial(n)
    num = np.zeros(2 * nf, dtype=np.uint64)
    den = np.zeros(2, dtype=np.uint64)
    unres = np.zeros(2, dtype=np.uint64)
    paths = ctypes.c_uint64(0)
    rc = _load().ms_oracle_enumerate_rs(n, B, max_levels, mode, num.ctypes.data,
                                        den.ctypes.data, ctypes.byref(paths), unres.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"ms_oracle_enumerate_rs failed with code {rc}")
    return _u128(num), _u128(den)[0], int(paths.value), _u128(unres)[0]
