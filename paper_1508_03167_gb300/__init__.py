"""GB300 MergeShuffle (arXiv 1508.03167): Python binding of libmergeshuffle.

The binding only marshals arguments: every step of the shuffle runs in the CUDA kernels of the
shared library (built in-tree for sm_103a; see ``_build.py``). PyTorch supplies device memory and
streams. The C entry points are exposed under their C names (``ms_shuffle``, ``ms_perm``, ...);
``shuffle_`` / ``perm`` / ``shuffle_host`` are conveniences over them for torch tensors.
There is no CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "MS_OK", "MS_ERR_INVALID", "MS_ERR_UNSUPPORTED", "MS_ERR_NOMEM", "MS_ERR_CUDA",
    "MS_ERR_TIMEOUT", "RANDOM_BIT_FIELDS", "ms_random_bits", "ms_random_bits_workspace", "random_bits", "MS_FLAG_TAIL_SEQUENTIAL", "MS_FLAG_PROFILE", "MS_FLAG_GLOBAL_LEVELS", "MS_FLAG_CTA_LEVELS", "MS_FLAG_PERM", "MS_FLAG_SINGLE_STREAM", "MS_FLAG_WARP_LEVELS", "MS_FLAG_SINGLE_LEVELS", "MS_FLAG_PAIR_LEVELS", "MS_FLAG_CTA_TILES", "MS_FLAG_LITERAL", "MS_FLAG_FDR", "MS_FLAG_BALANCED", "MS_MAX_B", "ms_batch_workspace_bytes",
    "ms_batch_prepare", "ms_batch_run", "ms_shuffle_batch", "batch_workspace", "shuffle_batch", "MsParams",
    "MsPlan", "MsProfile", "MsError", "ms_profile_read", "profile",
    "lib", "library_path", "ms_default_params", "ms_plan_info", "ms_workspace_bytes",
    "ms_shuffle", "ms_perm", "ms_host_workspace_bytes", "ms_shuffle_host", "ms_perm_host",
    "ms_status_string", "ms_version", "ms_last_cuda_error", "ms_perm_static", "MS_STATIC_MAX_N", "MS_STATIC_SCRATCH_BYTES", "params", "plan", "shuffle_", "perm", "shuffle_host",
    "perm_host", "workspace", "MsTuneEntry", "ms_resolve_params", "ms_resolve_batch_params",
    "ms_tune_install", "ms_tune_table", "resolve", "resolve_batch",
    "ms_rs_workspace_bytes", "ms_rs_shuffle", "ms_rs_perm", "rs_perm", "rs_shuffle_",
]

MS_OK, MS_ERR_INVALID, MS_ERR_UNSUPPORTED, MS_ERR_NOMEM, MS_ERR_CUDA, MS_ERR_TIMEOUT = range(6)
MS_FLAG_TAIL_SEQUENTIAL = 0x1
MS_FLAG_PROFILE = 0x2
MS_FLAG_GLOBAL_LEVELS = 0x4
MS_FLAG_CTA_LEVELS = 0x8
MS_FLAG_PERM = 0x10
MS_FLAG_SINGLE_STREAM = 0x20
MS_FLAG_WARP_LEVELS = 0x40
MS_FLAG_SINGLE_LEVELS = 0x80
MS_FLAG_PAIR_LEVELS = 0x100
MS_FLAG_CTA_TILES = 0x200
MS_FLAG_LITERAL = 0x400
MS_FLAG_FDR = 0x800
MS_FLAG_BALANCED = 0x1000
MS_MAX_B = 4096
MS_STATIC_MAX_N = 1 << 21
MS_STATIC_SCRATCH_BYTES = 16 << 20


class MsParams(ctypes.Structure):
    _fields_ = [("B", ctypes.c_uint32), ("fuse_depth", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("tile_bytes", ctypes.c_uint32)]


class MsPlan(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("w", ctypes.c_uint32), ("B", ctypes.c_uint32),
                ("c", ctypes.c_uint32), ("fuse_depth", ctypes.c_uint32),
                ("hbm_levels", ctypes.c_uint32), ("passes", ctypes.c_uint32),
                ("tiles", ctypes.c_uint64), ("tile_max", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_uint32),
                ("global_levels", ctypes.c_uint32), ("fused_pairs", ctypes.c_uint32),
                ("tile_smem", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class MsProfile(ctypes.Structure):
    _fields_ = [("kinds", ctypes.c_uint32), ("names", (ctypes.c_char * 24) * 16),
                ("launches", ctypes.c_uint64 * 16), ("ms", ctypes.c_double * 16)]

    def as_dict(self) -> dict:
        return {self.names[k].value.decode(): {"launches": int(self.launches[k]),
                                              "ms": float(self.ms[k])}
                for k in range(self.kinds)}


class MsTuneEntry(ctypes.Structure):
    _fields_ = [("w", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("log2n_max", ctypes.c_uint32), ("B", ctypes.c_uint32),
                ("fuse_depth", ctypes.c_int32), ("flags", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class MsError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = ""
        if status == MS_ERR_CUDA:
            code, text = ms_last_cuda_error()
            detail = f": CUDA error {code} ({text})"
        super().__init__(f"{what} failed: {ms_status_string(status)} ({status}){detail}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from . import _build

    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load (building first if needed) libmergeshuffle.so and declare its C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import _build

        path = _build.build()
        L = ctypes.CDLL(path)
        u32, u64, i32, sz, vp = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                 ctypes.c_size_t, ctypes.c_void_p)
        P = ctypes.POINTER(MsParams)
        L.ms_default_params.argtypes = [P]
        L.ms_default_params.restype = None
        L.ms_plan_info.argtypes = [u64, u32, P, ctypes.POINTER(MsPlan)]
        L.ms_plan_info.restype = i32
        L.ms_workspace_bytes.argtypes = [u64, u32, P]
        L.ms_workspace_bytes.restype = sz
        L.ms_shuffle.argtypes = [vp, u64, u32, u64, vp, sz, P, vp]
        L.ms_shuffle.restype = i32
        L.ms_perm.argtypes = [vp, u64, u64, vp, sz, P, vp]
        L.ms_perm.restype = i32
        L.ms_host_workspace_bytes.argtypes = [u64, u32, P]
        L.ms_host_workspace_bytes.restype = sz
        L.ms_shuffle_host.argtypes = [vp, u64, u32, u64, vp, sz, P, vp]
        L.ms_shuffle_host.restype = i32
        L.ms_perm_host.argtypes = [vp, u64, u64, vp, sz, P, vp]
        L.ms_perm_host.restype = i32
        pu64 = ctypes.POINTER(ctypes.c_uint64)
        pvp = ctypes.POINTER(ctypes.c_void_p)
        L.ms_batch_workspace_bytes.argtypes = [u32, pu64, u32, P]
        L.ms_batch_workspace_bytes.restype = sz
        for name in ("ms_batch_prepare", "ms_batch_run", "ms_shuffle_batch"):
            fn = getattr(L, name)
            fn.argtypes = [u32, pvp, pu64, u32, pu64, u64, vp, sz, P, vp]
            fn.restype = i32
        L.ms_resolve_params.argtypes = [u64, u32, P]
        L.ms_resolve_params.restype = i32
        L.ms_resolve_batch_params.argtypes = [u32, pu64, u32, P]
        L.ms_resolve_batch_params.restype = i32
        L.ms_tune_install.argtypes = [ctypes.POINTER(MsTuneEntry), u32]
        L.ms_tune_install.restype = i32
        L.ms_tune_table.argtypes = [ctypes.POINTER(MsTuneEntry), u32]
        L.ms_tune_table.restype = u32
        L.ms_perm_static.argtypes = [vp, u64, u64, P, vp]
        L.ms_perm_static.restype = i32
        L.ms_profile_read.argtypes = [ctypes.POINTER(MsProfile), i32]
        L.ms_profile_read.restype = i32
        L.ms_status_string.argtypes = [i32]
        L.ms_status_string.restype = ctypes.c_char_p
        L.ms_version.argtypes = []
        L.ms_version.restype = ctypes.c_char_p
        L.ms_random_bits_workspace.argtypes = [u64, P]
        L.ms_random_bits_workspace.restype = sz
        L.ms_random_bits.argtypes = [u64, u64, P, vp, sz, pu64, vp]
        L.ms_random_bits.restype = i32
        L.ms_rs_workspace_bytes.argtypes = [u64, u32, u32]
        L.ms_rs_workspace_bytes.restype = sz
        L.ms_rs_shuffle.argtypes = [vp, u64, u32, u64, u32, vp, sz, vp]
        L.ms_rs_shuffle.restype = i32
        L.ms_rs_perm.argtypes = [vp, u64, u64, u32, vp, sz, vp]
        L.ms_rs_perm.restype = i32
        L.ms_last_cuda_error.argtypes = []
        L.ms_last_cuda_error.restype = i32
        L.ms_last_cuda_error_string.argtypes = []
        L.ms_last_cuda_error_string.restype = ctypes.c_char_p
        _lib = L
        return L


# ------------------------------------------------------------------ C entry points ----------
def _p(p):
    return ctypes.byref(p) if p is not None else None


def ms_default_params() -> MsParams:
    p = MsParams()
    lib().ms_default_params(ctypes.byref(p))
    return p


def ms_plan_info(n: int, w: int, p: MsParams | None = None) -> MsPlan:
    out = MsPlan()
    st = lib().ms_plan_info(n, w, _p(p), ctypes.byref(out))
    if st != MS_OK:
        raise MsError(st, "ms_plan_info")
    return out


def ms_workspace_bytes(n: int, w: int, p: MsParams | None = None) -> int:
    return int(lib().ms_workspace_bytes(n, w, _p(p)))


def ms_host_workspace_bytes(n: int, w: int, p: MsParams | None = None) -> int:
    return int(lib().ms_host_workspace_bytes(n, w, _p(p)))


def ms_shuffle(d_data: int, n: int, w: int, seed: int, d_ws: int, ws_bytes: int,
               p: MsParams | None = None, stream: int = 0) -> int:
    return int(lib().ms_shuffle(d_data, n, w, seed, d_ws, ws_bytes, _p(p), stream))


def ms_perm(d_out: int, n: int, seed: int, d_ws: int, ws_bytes: int,
            p: MsParams | None = None, stream: int = 0) -> int:
    return int(lib().ms_perm(d_out, n, seed, d_ws, ws_bytes, _p(p), stream))


def ms_shuffle_host(h_data: int, n: int, w: int, seed: int, d_ws: int, ws_bytes: int,
                    p: MsParams | None = None, stream: int = 0) -> int:
    return int(lib().ms_shuffle_host(h_data, n, w, seed, d_ws, ws_bytes, _p(p), stream))


def ms_perm_host(h_out: int, n: int, seed: int, d_ws: int, ws_bytes: int,
                 p: MsParams | None = None, stream: int = 0) -> int:
    return int(lib().ms_perm_host(h_out, n, seed, d_ws, ws_bytes, _p(p), stream))


def _u64s(vals):
    if vals is None:
        return None
    vals = [int(v) for v in vals]
    return (ctypes.c_uint64 * max(len(vals), 1))(*vals)


def _ptrs(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_void_p * max(len(vals), 1))(*vals)


def ms_batch_workspace_bytes(ns, w: int, p: MsParams | None = None) -> int:
    return int(lib().ms_batch_workspace_bytes(len(ns), _u64s(ns), w, _p(p)))


def _batch_call(name, ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p, stream):
    k = len(ns)
    return int(getattr(lib(), name)(k, _ptrs(ptrs), _u64s(ns), w, _u64s(seeds), base_seed,
                                     d_ws, ws_bytes, _p(p), stream))


def ms_batch_prepare(ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p=None, stream=0) -> int:
    return _batch_call("ms_batch_prepare", ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p,
                       stream)


def ms_batch_run(ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p=None, stream=0) -> int:
    return _batch_call("ms_batch_run", ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p, stream)


def ms_shuffle_batch(ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p=None, stream=0) -> int:
    return _batch_call("ms_shuffle_batch", ptrs, ns, w, seeds, base_seed, d_ws, ws_bytes, p,
                       stream)


def ms_perm_static(d_out: int, n: int, seed: int, p: MsParams | None = None,
                   stream: int = 0) -> int:
    """ms_perm with the library's fixed 16 MiB device scratch (no workspace, no allocation)."""
    return int(lib().ms_perm_static(d_out, n, seed, _p(p), stream))


def ms_resolve_params(n: int, w: int, p: MsParams) -> MsParams:
    """Copy of p with B = 0 replaced by the autotuner table's choice for (n, w)."""
    out = MsParams(p.B, p.fuse_depth, p.flags, p.tile_bytes)
    st = lib().ms_resolve_params(n, w, ctypes.byref(out))
    if st != MS_OK:
        raise MsError(st, "ms_resolve_params")
    return out


def ms_resolve_batch_params(ns, w: int, p: MsParams) -> MsParams:
    out = MsParams(p.B, p.fuse_depth, p.flags, p.tile_bytes)
    st = lib().ms_resolve_batch_params(len(ns), _u64s(ns), w, ctypes.byref(out))
    if st != MS_OK:
        raise MsError(st, "ms_resolve_batch_params")
    return out


def ms_tune_install(entries) -> None:
    """Install a tuning table (a list of MsTuneEntry or dicts); an empty list restores the
    built-in table."""
    rows = [e if isinstance(e, MsTuneEntry) else MsTuneEntry(**e) for e in entries]
    arr = (MsTuneEntry * max(len(rows), 1))(*rows)
    st = lib().ms_tune_install(arr, len(rows))
    if st != MS_OK:
        raise MsError(st, "ms_tune_install")


def ms_tune_table() -> list[dict]:
    k = int(lib().ms_tune_table(None, 0))
    arr = (MsTuneEntry * max(k, 1))()
    k = int(lib().ms_tune_table(arr, k))
    return [arr[i].as_dict() for i in range(k)]


def ms_profile_read(reset: bool = True) -> MsProfile:
    out = MsProfile()
    st = lib().ms_profile_read(ctypes.byref(out), 1 if reset else 0)
    if st != MS_OK:
        raise MsError(st, "ms_profile_read")
    return out


def profile(reset: bool = True) -> dict:
    """Per-kernel-class launch counts and summed milliseconds of profiled calls."""
    return ms_profile_read(reset).as_dict()


def ms_status_string(st: int) -> str:
    return lib().ms_status_string(st).decode()


def ms_version() -> str:
    return lib().ms_version().decode()


RANDOM_BIT_FIELDS = ("coin_bits", "leaf_bits", "tail_bits", "leaf_draws", "tail_draws",
                     "merges", "leftover", "levels")


def ms_random_bits_workspace(n: int, p: MsParams | None = None) -> int:
    return int(lib().ms_random_bits_workspace(n, _p(p)))


def ms_random_bits(n: int, seed: int, d_ws: int, ws_bytes: int, p: MsParams | None = None,
                   stream: int = 0) -> dict:
    """Random bits consumed by ms_perm(n, seed) with parameters p (see the header)."""
    out = (ctypes.c_uint64 * 8)()
    st = lib().ms_random_bits(n, seed, _p(p), d_ws, ws_bytes, out, stream)
    if st != MS_OK:
        raise MsError(st, "ms_random_bits")
    d = {k: int(v) for k, v in zip(RANDOM_BIT_FIELDS, out)}
    d["total_bits"] = d["coin_bits"] + d["leaf_bits"] + d["tail_bits"]
    return d


def random_bits(n: int, seed: int, device=None, **kw) -> dict:
    """ms_random_bits with a workspace allocated by PyTorch on `device` (default cuda:0)."""
    import torch

    p = params(**kw)
    dev = torch.device(device) if device is not None else torch.device("cuda")
    nbytes = ms_random_bits_workspace(n, p)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
    return ms_random_bits(n, seed, ws.data_ptr(), nbytes, p,
                          torch.cuda.current_stream(dev).cuda_stream)


def ms_last_cuda_error() -> tuple[int, str]:
    """The CUDA error behind this thread's last MS_ERR_CUDA (code, description)."""
    return int(lib().ms_last_cuda_error()), lib().ms_last_cuda_error_string().decode()


# ------------------------------------------------------------------ torch conveniences -------
def params(B: int = 1024, fuse_depth: int = -1, flags: int = 0, tile_bytes: int = 0) -> MsParams:
    return MsParams(B, fuse_depth, flags, tile_bytes)


def plan(n: int, w: int = 4, **kw) -> dict:
    return ms_plan_info(n, w, params(**kw)).as_dict()


def resolve(n: int, w: int = 4, **kw) -> MsParams:
    """Parameters a call on (n, w) runs with: B = 0 (autotuned) resolved by the tuning table."""
    return ms_resolve_params(n, w, params(**kw))


def resolve_batch(ns, w: int = 4, **kw) -> MsParams:
    return ms_resolve_batch_params(list(ns), w, params(**kw))


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _width(x) -> tuple[int, int]:
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    n = x.shape[0] if x.dim() > 0 else 0
    if n == 0:
        return 0, 4
    w = x.numel() * x.element_size() // n
    return n, w


def workspace(n: int, w: int = 4, device=None, host: bool = False, **kw):
    """Allocate a device workspace (torch's caching allocator) for a call with these sizes."""
    import torch

    p = params(**kw)
    nbytes = ms_host_workspace_bytes(n, w, p) if host else ms_workspace_bytes(n, w, p)
    if nbytes == 0:
        raise MsError(MS_ERR_INVALID, "workspace sizing")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def shuffle_(x, seed: int, B: int = 1024, fuse_depth: int = -1, flags: int = 0,
             tile_bytes: int = 0, ws=None, stream=None):
    """Permute the rows of a contiguous CUDA tensor in place (rows of 1, 2, 4, 8 or 16 bytes)."""
    n, w = _width(x)
    p = params(B, fuse_depth, flags, tile_bytes)
    if n == 0:
        return x
    if ws is None:
        ws = workspace(n, w, x.device, B=B, fuse_depth=fuse_depth, flags=flags,
                       tile_bytes=tile_bytes)
    st = ms_shuffle(x.data_ptr(), n, w, seed, ws.data_ptr(), ws.numel(), p, _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_shuffle")
    return x


def perm(n: int, seed: int, B: int = 1024, fuse_depth: int = -1, flags: int = 0,
         tile_bytes: int = 0, device=None, out=None, ws=None, stream=None):
    """A uniformly random permutation of 0..n-1 as an int32 CUDA tensor (uint32 bit pattern)."""
    import torch

    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=device or "cuda")
    p = params(B, fuse_depth, flags, tile_bytes)
    if ws is None:
        ws = workspace(n, 4, out.device, B=B, fuse_depth=fuse_depth, flags=flags,
                       tile_bytes=tile_bytes)
    st = ms_perm(out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(), p, _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_perm")
    return out


def shuffle_host(h, seed: int, ws, B: int = 1024, fuse_depth: int = -1, flags: int = 0,
                 tile_bytes: int = 0, stream=None):
    """Shuffle a contiguous host tensor (ideally pinned) through the device; synchronous."""
    n, w = _width(h)
    st = ms_shuffle_host(h.data_ptr(), n, w, seed, ws.data_ptr(), ws.numel(),
                         params(B, fuse_depth, flags, tile_bytes), _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_shuffle_host")
    return h


def perm_host(h_out, seed: int, ws, B: int = 1024, fuse_depth: int = -1, flags: int = 0,
              tile_bytes: int = 0, stream=None):
    n = h_out.shape[0]
    st = ms_perm_host(h_out.data_ptr(), n, seed, ws.data_ptr(), ws.numel(),
                      params(B, fuse_depth, flags, tile_bytes), _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_perm_host")
    return h_out


def batch_workspace(ns, w: int = 4, device=None, **kw):
    import torch

    nbytes = ms_batch_workspace_bytes(list(ns), w, params(**kw))
    if nbytes == 0:
        raise MsError(MS_ERR_INVALID, "batch workspace sizing")
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def shuffle_batch(tensors, base_seed: int = 0, seeds=None, perm: bool = False, B: int = 1024,
                  fuse_depth: int = -1, flags: int = 0, ws=None, stream=None):
    """Shuffle (or, with perm=True, fill with permutations) a list of contiguous CUDA tensors,
    instance i with seed seeds[i] or base_seed + i."""
    widths = set()
    ns, ptrs = [], []
    for t in tensors:
        n, w = _width(t)
        ns.append(n)
        ptrs.append(t.data_ptr() if n else 0)
        if n:
            widths.add(w)
    if len(widths) > 1:
        raise ValueError("all instances must have the same element width")
    w = widths.pop() if widths else 4
    fl = flags | (MS_FLAG_PERM if perm else 0)
    p = params(B, fuse_depth, fl)
    if ws is None:
        ws = batch_workspace(ns, w, tensors[0].device if tensors else None, B=B,
                             fuse_depth=fuse_depth, flags=fl)
    st = ms_shuffle_batch(ptrs, ns, w, seeds, base_seed, ws.data_ptr(), ws.numel(), p,
                          _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_shuffle_batch")
    return tensors


# ------------------------------------------------------------------ splitting process -------
def ms_rs_workspace_bytes(n: int, w: int, B: int) -> int:
    return int(lib().ms_rs_workspace_bytes(n, w, B))


def ms_rs_shuffle(d_data: int, n: int, w: int, seed: int, B: int, d_ws: int, ws_bytes: int,
                  stream: int = 0) -> int:
    return int(lib().ms_rs_shuffle(d_data, n, w, seed, B, d_ws, ws_bytes, stream))


def ms_rs_perm(d_out: int, n: int, seed: int, B: int, d_ws: int, ws_bytes: int,
               stream: int = 0) -> int:
    return int(lib().ms_rs_perm(d_out, n, seed, B, d_ws, ws_bytes, stream))


def rs_perm(n: int, seed: int, B: int, device=None, out=None, stream=None):
    """The Rao-Sandelius splitting process's permutation of 0..n-1 (int32 CUDA tensor)."""
    import torch

    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=device or "cuda")
    nbytes = ms_rs_workspace_bytes(n, 4, B)
    if nbytes == 0:
        raise MsError(MS_ERR_INVALID, "ms_rs_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=out.device)
    st = ms_rs_perm(out.data_ptr(), n, seed, B, ws.data_ptr(), nbytes, _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_rs_perm")
    return out


def rs_shuffle_(x, seed: int, B: int, stream=None):
    """Shuffle a contiguous CUDA tensor in place along its first axis by the splitting process."""
    import torch

    n, w = _width(x)
    nbytes = ms_rs_workspace_bytes(n, w, B)
    if nbytes == 0:
        raise MsError(MS_ERR_INVALID, "ms_rs_workspace_bytes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    st = ms_rs_shuffle(x.data_ptr(), n, w, seed, B, ws.data_ptr(), nbytes, _stream_handle(stream))
    if st != MS_OK:
        raise MsError(st, "ms_rs_shuffle")
    return x
