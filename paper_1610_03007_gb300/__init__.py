"""gbsa — suffix arrays on one GB300 by prefix doubling with discarding.

Thin ctypes binding over the C-ABI of libgbsa.so (include/gbsa.h): it only
marshals arguments. Every step of the method runs in the library's CUDA
kernels; PyTorch supplies device memory and the current stream. There is no
CPU fallback: if libgbsa.so is missing or no GPU is present, the calls raise.

Method: Bingmann, Gog & Kurpicz, "Scalable Construction of Text Indexes"
(arXiv 1610.03007), Section 2.1, Algorithms 1, 4 and 5.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbsa.so")

SA_OK = 0
STATUS_NAMES = {0: "SA_OK", 1: "SA_ERR_INVALID_ARG", 2: "SA_ERR_TOO_LARGE", 3: "SA_ERR_OOM",
                4: "SA_ERR_CUDA", 5: "SA_ERR_TIMEOUT", 6: "SA_ERR_INTERNAL"}
SA_ERR_TIMEOUT = 5
SA_MAX_N = 1 << 31
SA_MAX_ROUNDS = 64

# Symbols include/gbsa.h declares; the loader checks that all are exported.
EXPORTED = ("sa_build", "sa_workspace_bytes", "sa_build_ex", "sa_build_batched",
            "sa_batched_workspace_bytes", "sa_build_batched_ex", "sa_build_host", "sa_build_batched_host",
            "sa_sort_pairs", "sa_sort_workspace_bytes", "sa_status_string",
            "sa_build_noalloc", "sa_request_footprint", "sa_server_create", "sa_server_submit",
            "sa_server_poll", "sa_server_wait", "sa_server_get_stats", "sa_server_destroy",
            "sa_bwt", "sa_lcp", "sa_lcp_workspace_bytes", "sa_build_dc3", "sa_build_dc7",
            "sa_build_pd_sort", "sa_pool_usage", "sa_tuning_set", "sa_tuning_load",
            "sa_tuning_lookup", "sa_pool_trim")


class SAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class Options(ctypes.Structure):
    _fields_ = [("h0_chars", ctypes.c_uint32), ("spin_limit", ctypes.c_uint32),
                ("inject_stall", ctypes.c_uint32), ("trace_isa", ctypes.c_void_p),
                ("trace_cap", ctypes.c_uint32), ("paper_names", ctypes.c_uint32),
                ("refine_shape", ctypes.c_uint32), ("sort_items", ctypes.c_uint32),
                ("profile", ctypes.c_uint32), ("multiplier", ctypes.c_uint32),
                ("bucket_min", ctypes.c_uint32), ("device_rounds", ctypes.c_uint32),
                ("group_order", ctypes.c_uint32), ("initial_keys", ctypes.c_uint32)]


class Tuned(ctypes.Structure):
    """One entry of the library's tuning table (sa_tuned)."""
    _fields_ = [("sort_items", ctypes.c_uint32), ("refine_shape", ctypes.c_uint32),
                ("h0_chars", ctypes.c_uint32), ("bucket_min", ctypes.c_uint32)]

    def to_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


KERNEL_CLASSES = ("byte_hist", "pack", "digit_hist", "plan", "onesweep", "rename", "gather",
                  "output", "refine", "scatter", "classify", "apply", "bucket", "reorder")


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("sigma", ctypes.c_uint32),
                ("bits_per_char", ctypes.c_uint32), ("chars_per_key", ctypes.c_uint32),
                ("active", ctypes.c_uint64 * SA_MAX_ROUNDS),
                ("unique", ctypes.c_uint64 * SA_MAX_ROUNDS),
                ("passes", ctypes.c_uint32 * SA_MAX_ROUNDS),
                ("key_bits", ctypes.c_uint32 * SA_MAX_ROUNDS),
                ("groups", ctypes.c_uint64 * SA_MAX_ROUNDS),
                ("bytes_model", ctypes.c_uint64),
                ("launches", ctypes.c_uint32),
                ("kernel_ms", ctypes.c_double * len(KERNEL_CLASSES)),
                ("kernel_launches", ctypes.c_uint64 * len(KERNEL_CLASSES)),
                ("kernel_bytes", ctypes.c_uint64 * len(KERNEL_CLASSES)),
                ("sort_items", ctypes.c_uint32), ("refine_shape", ctypes.c_uint32),
                ("bucket_min", ctypes.c_uint32), ("tuned", ctypes.c_uint32)]

    def to_dict(self) -> dict:
        r = self.rounds
        return {"rounds": r, "sigma": self.sigma, "bits_per_char": self.bits_per_char,
                "chars_per_key": self.chars_per_key,
                "active": list(self.active[:r]), "unique": list(self.unique[:r]),
                "passes": list(self.passes[:r]), "key_bits": list(self.key_bits[:r]),
                "groups": list(self.groups[:r]), "bytes_model": int(self.bytes_model),
                "launches": int(self.launches),
                "params": {"sort_items": int(self.sort_items),
                           "refine_shape": int(self.refine_shape),
                           "h0_chars": int(self.chars_per_key),
                           "bucket_min": int(self.bucket_min),
                           "from_table": bool(self.tuned)},
                "kernels": {name: {"ms": self.kernel_ms[k], "launches": int(self.kernel_launches[k]),
                                   "bytes": int(self.kernel_bytes[k])}
                            for k, name in enumerate(KERNEL_CLASSES)}}


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("device", ctypes.c_int32), ("simulate", ctypes.c_uint32),
                ("simulate_ns_per_byte", ctypes.c_double), ("size_priority", ctypes.c_uint32),
                ("merge_requests", ctypes.c_uint32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_uint64), ("slot", ctypes.c_uint32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("priority", ctypes.c_int32),
                ("batch", ctypes.c_uint32)]

    def to_dict(self) -> dict:
        return {"status": self.status, "n": self.n, "slot": self.slot,
                "submit_s": self.submit_s, "start_s": self.start_s, "done_s": self.done_s,
                "latency_s": self.done_s - self.submit_s, "priority": self.priority,
                "batch": self.batch}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes_in_use", ctypes.c_uint64),
                ("in_flight", ctypes.c_uint32), ("peak_in_flight", ctypes.c_uint32),
                ("queued", ctypes.c_uint32), ("tracked", ctypes.c_uint32),
                ("builds", ctypes.c_uint64), ("merged", ctypes.c_uint64)]


_lib = None


def load(path: str | None = None):
    """Load libgbsa.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"gbsa CUDA library not built: {p} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(p)
    missing = [s for s in EXPORTED if not hasattr(lib, s)]
    if missing:
        raise RuntimeError(f"{p} lacks symbols {missing}")
    vp, u64, u32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t
    lib.sa_build.argtypes = [vp, u64, vp, vp]
    lib.sa_workspace_bytes.argtypes = [u64]
    lib.sa_workspace_bytes.restype = sz
    lib.sa_build_ex.argtypes = [vp, u64, vp, vp, vp, sz, ctypes.POINTER(Options),
                                ctypes.POINTER(Stats), vp]
    lib.sa_build_batched.argtypes = [vp, vp, u32, vp, vp]
    lib.sa_batched_workspace_bytes.argtypes = [vp, u32]
    lib.sa_batched_workspace_bytes.restype = sz
    lib.sa_build_batched_ex.argtypes = [vp, vp, u32, vp, vp, sz, ctypes.POINTER(Options),
                                        ctypes.POINTER(Stats), vp]
    lib.sa_build_host.argtypes = [vp, u64, vp, vp]
    lib.sa_build_batched_host.argtypes = [vp, vp, vp, u32, vp]
    lib.sa_build_noalloc.argtypes = [vp, u64, vp, vp]
    lib.sa_sort_pairs.argtypes = [vp, vp, u64, u32, u32, vp, sz, vp]
    lib.sa_bwt.argtypes = [vp, u64, vp, vp, vp, vp]
    lib.sa_build_dc3.argtypes = [vp, u64, vp, vp, vp]
    lib.sa_build_dc7.argtypes = [vp, u64, vp, vp, vp]
    lib.sa_build_pd_sort.argtypes = [vp, u64, vp, vp, u32, vp, vp]
    lib.sa_lcp.argtypes = [vp, u64, vp, vp, vp, sz, vp]
    lib.sa_lcp_workspace_bytes.argtypes = [u64]
    lib.sa_lcp_workspace_bytes.restype = sz
    lib.sa_sort_workspace_bytes.argtypes = [u64]
    lib.sa_sort_workspace_bytes.restype = sz
    lib.sa_request_footprint.argtypes = [u64]
    lib.sa_request_footprint.restype = sz
    lib.sa_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.sa_server_create.restype = ctypes.c_int
    lib.sa_server_submit.argtypes = [vp, vp, u64, vp, ctypes.POINTER(u64)]
    lib.sa_server_submit.restype = ctypes.c_int
    lib.sa_server_poll.argtypes = [vp, u64, ctypes.POINTER(RequestInfo)]
    lib.sa_server_poll.restype = ctypes.c_int
    lib.sa_server_wait.argtypes = [vp, u64, ctypes.POINTER(RequestInfo)]
    lib.sa_server_wait.restype = ctypes.c_int
    lib.sa_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.sa_server_get_stats.restype = None
    lib.sa_server_destroy.argtypes = [vp]
    lib.sa_server_destroy.restype = None
    lib.sa_tuning_set.argtypes = [u32, u32, u32, ctypes.POINTER(Tuned)]
    lib.sa_tuning_set.restype = ctypes.c_int
    lib.sa_tuning_load.argtypes = [ctypes.c_char_p]
    lib.sa_tuning_load.restype = ctypes.c_int
    lib.sa_tuning_lookup.argtypes = [u32, u32, u64, ctypes.POINTER(Tuned)]
    lib.sa_tuning_lookup.restype = u32
    lib.sa_pool_trim.argtypes = [u64]
    lib.sa_pool_trim.restype = ctypes.c_int
    lib.sa_pool_usage.argtypes = [ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.sa_pool_usage.restype = ctypes.c_int
    lib.sa_status_string.argtypes = [ctypes.c_int]
    lib.sa_status_string.restype = ctypes.c_char_p
    for f in ("sa_build", "sa_build_ex", "sa_build_batched", "sa_build_batched_ex",
              "sa_build_host", "sa_build_batched_host", "sa_sort_pairs", "sa_build_noalloc"):
        getattr(lib, f).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def tuning_set(batched: int, bits_per_char: int, log2_n: int, params: dict | None):
    """Set (or, with params None, remove) one entry of the library's tuning
    table (sa_tuning_set); params holds any of sort_items, refine_shape,
    h0_chars, bucket_min."""
    lib = load()
    t = Tuned(**params) if params is not None else None
    _check(lib.sa_tuning_set(batched, bits_per_char, log2_n,
                             ctypes.byref(t) if t is not None else None), "sa_tuning_set")


def tuning_load(path: str | None):
    """Replace the library's tuning table by a table file (None: empty)."""
    lib = load()
    _check(lib.sa_tuning_load(path.encode() if path else None), "sa_tuning_load")


def tuning_lookup(batched: int, bits_per_char: int, n: int) -> tuple[dict, int]:
    """(the parameters a build of this class would take from the table,
    number of table entries)."""
    lib = load()
    t = Tuned()
    count = lib.sa_tuning_lookup(batched, bits_per_char, n, ctypes.byref(t))
    return t.to_dict(), int(count)


def pool_usage() -> tuple[int, int]:
    """(used, reserved) bytes of the library's device memory pool on the
    current device (sa_pool_usage)."""
    lib = load()
    u, r = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.sa_pool_usage(ctypes.byref(u), ctypes.byref(r)), "sa_pool_usage")
    return int(u.value), int(r.value)


def pool_trim(keep_bytes: int = 0):
    """Give the library pool's unused device memory back (sa_pool_trim)."""
    _check(load().sa_pool_trim(keep_bytes), "sa_pool_trim")


def _torch():
    import torch
    return torch


def _stream(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(status: int, where: str):
    if status != SA_OK:
        raise SAError(status, where)


def _dev_u8(t):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.dim() == 1):
        raise TypeError("text must be a 1-D torch.uint8 CUDA tensor")
    return t.contiguous()


def _dev_buf(x, name: str, device, itemsize: int, at_least: int):
    """x, if it is a contiguous CUDA tensor on `device` holding at least
    `at_least` elements of `itemsize` bytes: the library reads or writes that
    many elements from the first one, so any other buffer could take a
    kernel past its end."""
    torch = _torch()
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.device == device
            and x.is_contiguous() and x.element_size() == itemsize and x.numel() >= at_least):
        raise ValueError(f"{name} must be a contiguous CUDA tensor on {device} with at least "
                         f"{at_least} elements of {itemsize} bytes")
    return x


def _dev_ws(x, device):
    """(pointer, bytes) of a caller's workspace, a contiguous CUDA tensor on
    `device` (the library checks the size); (None, 0) for None."""
    torch = _torch()
    if x is None:
        return None, 0
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.device == device
            and x.is_contiguous()):
        raise ValueError(f"workspace must be a contiguous CUDA tensor on {device}")
    return x.data_ptr(), x.numel() * x.element_size()


def _host_out(x, n: int, name: str):
    """x, if it is a writable C-contiguous numpy array of n elements of 4
    bytes (the library writes n uint32 from its first one)."""
    if not (isinstance(x, np.ndarray) and x.itemsize == 4 and x.size == n
            and x.flags.c_contiguous and x.flags.writeable):
        raise ValueError(f"{name} must be a writable C-contiguous numpy array of {n} "
                         "4-byte elements")
    return x


def workspace_bytes(n: int) -> int:
    return int(load().sa_workspace_bytes(n))


def sa_build(text, sa_out=None, stream=None):
    """SA of one text (torch uint8 CUDA tensor). Returns int32 (uint32 bits)."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    if sa_out is None:
        sa_out = torch.empty(n, dtype=torch.int32, device=t.device)
    _dev_buf(sa_out, "sa_out", t.device, 4, n)
    _check(lib.sa_build(t.data_ptr(), n, sa_out.data_ptr() if n else None, _stream(stream)),
           "sa_build")
    return sa_out


def sa_build_ex(text, *, isa=False, workspace=None, h0_chars=0, spin_limit=0,
                inject_stall=0, trace_cap=0, paper_names=False, refine_shape=0, sort_items=0,
                profile=False, multiplier=0, bucket_min=0, device_rounds=0, group_order=0,
                initial_keys=0, stream=None):
    """sa_build with options. Returns (sa, isa or None, stats dict, trace or None).

    multiplier: growth factor a of the resolved prefix per round (0 or 2:
    doubling; 3, 4: tripling, quadrupling). initial_keys: 0 or 1 = formed
    inside the first radix pass where that applies, 2 = by a separate pack.

    workspace: a uint8 CUDA tensor of at least workspace_bytes(n) bytes, or
    None to let torch's caching allocator provide one."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    dev = t.device
    sa = torch.empty(n, dtype=torch.int32, device=dev)
    isa_t = torch.empty(n, dtype=torch.int32, device=dev) if isa else None
    wsb = int(lib.sa_workspace_bytes(n))
    if workspace is None:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ws_ptr, ws_bytes = _dev_ws(workspace, dev)
    trace = torch.zeros((trace_cap, n), dtype=torch.int32, device=dev) if trace_cap else None
    opt = Options(h0_chars, spin_limit, inject_stall,
                  trace.data_ptr() if trace is not None and n else None, trace_cap,
                  1 if paper_names else 0, refine_shape, sort_items, 1 if profile else 0,
                  multiplier, bucket_min, device_rounds, group_order, initial_keys)
    st = Stats()
    rc = lib.sa_build_ex(t.data_ptr(), n, sa.data_ptr() if n else None,
                         isa_t.data_ptr() if isa_t is not None and n else None,
                         ws_ptr, ws_bytes, ctypes.byref(opt),
                         ctypes.byref(st), _stream(stream))
    _check(rc, "sa_build_ex")
    return sa, isa_t, st.to_dict(), trace


def sa_build_batched(texts, offsets, sa_out=None, workspace=None, stream=None, stats=False,
                     profile=False, refine_shape=0, sort_items=0, h0_chars=0, multiplier=0,
                     bucket_min=0, device_rounds=0, group_order=0):
    """SAs of many texts in one launch sequence.

    texts: 1-D uint8 CUDA tensor (the texts concatenated); offsets: host
    sequence of count+1 byte offsets. Returns int32 SAs with local indices at
    the same offsets (and the stats dict when stats=True)."""
    torch = _torch()
    lib = load()
    t = _dev_u8(texts)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    count = off.size - 1
    N = int(off[-1]) if count >= 0 else 0
    if sa_out is None:
        sa_out = torch.empty(N, dtype=torch.int32, device=t.device)
    _dev_buf(sa_out, "sa_out", t.device, 4, N)
    wsb = int(lib.sa_batched_workspace_bytes(off.ctypes.data, count))
    if workspace is None and N:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=t.device)
    ws_ptr, ws_bytes = _dev_ws(workspace, t.device)
    st = Stats()
    opt = Options(h0_chars, 0, 0, None, 0, 0, refine_shape, sort_items, 1 if profile else 0,
                  multiplier, bucket_min, device_rounds, group_order)
    rc = lib.sa_build_batched_ex(t.data_ptr(), off.ctypes.data, count,
                                 sa_out.data_ptr() if N else None, ws_ptr, ws_bytes,
                                 ctypes.byref(opt), ctypes.byref(st), _stream(stream))
    _check(rc, "sa_build_batched")
    return (sa_out, st.to_dict()) if stats else sa_out


def sa_build_host(text: np.ndarray, sa_out: np.ndarray | None = None, stream=None) -> np.ndarray:
    """End-to-end build from host memory (host text in, host SA out)."""
    lib = load()
    a = np.ascontiguousarray(text, dtype=np.uint8)
    if sa_out is None:
        sa_out = np.empty(a.size, dtype=np.uint32)
    _host_out(sa_out, a.size, "sa_out")
    _check(lib.sa_build_host(a.ctypes.data, a.size, sa_out.ctypes.data, _stream(stream)),
           "sa_build_host")
    return sa_out


def sa_build_host_ptr(host_text_ptr: int, n: int, host_sa_ptr: int, stream=None):
    """sa_build_host on raw (e.g. pinned torch) host pointers."""
    _check(load().sa_build_host(host_text_ptr, n, host_sa_ptr, _stream(stream)), "sa_build_host")


def sa_build_batched_host(texts, outs=None, stream=None) -> list:
    """sa_build_host for several host texts built as one batch: texts is a
    sequence of uint8 numpy arrays (or objects with .ctypes, e.g. pinned
    torch tensors' numpy views); returns one uint32 SA per text (outs, when
    given, are filled instead)."""
    lib = load()
    arrs = [np.ascontiguousarray(t, dtype=np.uint8) for t in texts]
    if outs is None:
        outs = [np.empty(a.size, dtype=np.uint32) for a in arrs]
    count = len(arrs)
    if len(outs) != count:
        raise ValueError("one output array per text")
    for k, (a, o) in enumerate(zip(arrs, outs)):
        _host_out(o, a.size, f"outs[{k}]")
    tp = (ctypes.c_void_p * max(count, 1))(*[a.ctypes.data if a.size else None for a in arrs])
    sp = (ctypes.c_void_p * max(count, 1))(*[o.ctypes.data if o.size else None for o in outs])
    ln = (ctypes.c_uint64 * max(count, 1))(*[a.size for a in arrs])
    _check(lib.sa_build_batched_host(tp, ln, sp, count, _stream(stream)), "sa_build_batched_host")
    return outs


def sa_sort_pairs(keys, vals, begin_bit=0, end_bit=64, workspace=None, stream=None):
    """Stable in-place LSD radix sort of (int64 keys as uint64, int32 vals as
    uint32) CUDA tensors by key bits [begin_bit, end_bit)."""
    torch = _torch()
    lib = load()
    if not (isinstance(keys, torch.Tensor) and keys.is_cuda):
        raise ValueError("keys must be a CUDA tensor")
    m = keys.numel()
    _dev_buf(keys, "keys", keys.device, 8, m)
    _dev_buf(vals, "vals", keys.device, 4, m)
    if vals.numel() != m:
        raise ValueError("keys and vals must have the same length")
    if workspace is None and m > 1:
        workspace = torch.empty(int(lib.sa_sort_workspace_bytes(m)), dtype=torch.uint8,
                                device=keys.device)
    ws_ptr, ws_bytes = _dev_ws(workspace, keys.device)
    _check(lib.sa_sort_pairs(keys.data_ptr(), vals.data_ptr(), m, begin_bit, end_bit,
                             ws_ptr, ws_bytes, _stream(stream)), "sa_sort_pairs")
    return keys, vals


def sa_bwt(text, sa, stream=None):
    """Burrows-Wheeler transform of text$ from its suffix array (CUDA uint8
    and int32 tensors). Returns (bwt uint8 tensor of n + 1 rows, primary
    index); the $ is stored as 0 at the primary row."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    _dev_buf(sa, "sa", t.device, 4, n)
    bwt = torch.empty(n + 1, dtype=torch.uint8, device=t.device)
    prim = torch.zeros(1, dtype=torch.int64, device=t.device)
    _check(lib.sa_bwt(t.data_ptr() if n else None, n, sa.data_ptr() if n else None,
                      bwt.data_ptr(), prim.data_ptr(), _stream(stream)), "sa_bwt")
    return bwt, int(prim.item())


def sa_build_dc3(text, trace=False, stream=None):
    """Suffix array by DC3 (the skew algorithm). Returns the int32 SA, and
    with trace=True also the top level's recursion string (1-based names of
    the triples at positions 1 mod 3, then 2 mod 3)."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    sa = torch.empty(n, dtype=torch.int32, device=t.device)
    tr = None
    if trace:
        tr = torch.zeros(max((n + 2) // 3 + n // 3, 1), dtype=torch.int32, device=t.device)
    _check(lib.sa_build_dc3(t.data_ptr() if n else None, n, sa.data_ptr() if n else None,
                            tr.data_ptr() if tr is not None else None, _stream(stream)),
           "sa_build_dc3")
    return (sa, tr) if trace else sa


def sa_build_dc7(text, trace=False, stream=None):
    """Suffix array by DC7 (difference cover {0, 1, 3} modulo 7). Returns
    the int32 SA, and with trace=True also the top level's recursion string
    (1-based names of the 7-character windows at positions 0, then 1, then
    3 mod 7, each class up to and including position n)."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    sa = torch.empty(n, dtype=torch.int32, device=t.device)
    tr = None
    if trace:
        m = sum((n - a) // 7 + 1 for a in (0, 1, 3) if a <= n)
        tr = torch.zeros(max(m, 1), dtype=torch.int32, device=t.device)
    _check(lib.sa_build_dc7(t.data_ptr() if n else None, n, sa.data_ptr() if n else None,
                            tr.data_ptr() if tr is not None else None, _stream(stream)),
           "sa_build_dc7")
    return (sa, tr) if trace else sa


def sa_build_pd_sort(text, trace_cap=0, stream=None):
    """Suffix array by prefix doubling using sorting (no discarding; the
    partner names by a sort with Eq. 1's comparator). Returns (sa, trace,
    rounds): trace[r] holds every position's name after the r-th naming
    (None when trace_cap = 0), rounds the number of namings."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    sa = torch.empty(n, dtype=torch.int32, device=t.device)
    tr = torch.zeros((trace_cap, n), dtype=torch.int32, device=t.device) if trace_cap else None
    rounds = ctypes.c_uint32(0)
    _check(lib.sa_build_pd_sort(t.data_ptr() if n else None, n, sa.data_ptr() if n else None,
                                tr.data_ptr() if tr is not None and n else None, trace_cap,
                                ctypes.byref(rounds), _stream(stream)),
           "sa_build_pd_sort")
    return sa, tr, int(rounds.value)


def sa_lcp(text, sa, workspace=None, stream=None):
    """LCP array of text from its suffix array (CUDA uint8 and int32
    tensors): int32 tensor, lcp[0] = 0, lcp[j] = longest common prefix of
    the suffixes sa[j-1] and sa[j]."""
    torch = _torch()
    lib = load()
    t = _dev_u8(text)
    n = t.numel()
    _dev_buf(sa, "sa", t.device, 4, n)
    lcp = torch.empty(n, dtype=torch.int32, device=t.device)
    if n and workspace is None:
        workspace = torch.empty(int(lib.sa_lcp_workspace_bytes(n)), dtype=torch.uint8,
                                device=t.device)
    ws_ptr, ws_bytes = _dev_ws(workspace, t.device)
    _check(lib.sa_lcp(t.data_ptr() if n else None, n, sa.data_ptr() if n else None,
                      lcp.data_ptr() if n else None, ws_ptr, ws_bytes, _stream(stream)),
           "sa_lcp")
    return lcp


def status_string(s: int) -> str:
    return load().sa_status_string(s).decode()


class Server:
    """Continuous-batching SA server (sa_server_* in include/gbsa.h).

    submit() takes a host numpy uint8 text and returns a ticket; the output
    buffer (numpy uint32) is kept alive here until the request is waited on.
    size_priority: smaller requests run on higher-priority CUDA streams
    (sa_server_config.size_priority); the info dict reports the priority.
    merge_requests: most queued small requests one build takes
    (sa_server_config.merge_requests; 0 or 1 = none merged, the default);
    the info dict reports the batch size.
    """

    def __init__(self, budget_bytes: int = 0, slots: int = 0, device: int = -1,
                 simulate_ns_per_byte: float = 0.0, size_priority: bool = True,
                 merge_requests: int = 0):
        self._lib = load()
        cfg = ServerConfig(budget_bytes, slots, device, 1 if simulate_ns_per_byte > 0 else 0,
                           simulate_ns_per_byte, 0 if size_priority else 1, merge_requests)
        h = ctypes.c_void_p()
        _check(self._lib.sa_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sa_server_create")
        self._h = h
        self._keep = {}

    def submit(self, text: np.ndarray, out: np.ndarray | None = None) -> int:
        a = np.ascontiguousarray(text, dtype=np.uint8)
        if out is None:
            out = np.empty(a.size, dtype=np.uint32)
        _host_out(out, a.size, "out")
        t = ctypes.c_uint64()
        _check(self._lib.sa_server_submit(self._h, a.ctypes.data, a.size, out.ctypes.data,
                                          ctypes.byref(t)), "sa_server_submit")
        self._keep[t.value] = (a, out)
        return t.value

    def poll(self, ticket: int):
        """None while the request runs; once done, (SA, info dict) as wait()
        returns them (the server then forgets the ticket)."""
        info = RequestInfo()
        r = self._lib.sa_server_poll(self._h, ticket, ctypes.byref(info))
        if r != 1:
            return None
        _, out = self._keep.pop(ticket)
        _check(info.status, "sa_server request")
        return out, info.to_dict()

    def wait(self, ticket: int):
        """(SA as numpy uint32, info dict); raises SAError if the build failed."""
        info = RequestInfo()
        st = self._lib.sa_server_wait(self._h, ticket, ctypes.byref(info))
        _, out = self._keep.pop(ticket)
        _check(st, "sa_server request")
        return out, info.to_dict()

    def stats(self) -> dict:
        s = ServerStats()
        self._lib.sa_server_get_stats(self._h, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            self._lib.sa_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
