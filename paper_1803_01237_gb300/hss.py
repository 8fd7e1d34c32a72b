"""Thin ctypes binding of libhss.so (include/hss.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (device memory and the current
stream come from torch); 64-bit keys travel as torch.int64 tensors whose bits
are either unsigned (key_type="u64") or signed (key_type="i64").  There is no
CPU fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhss.so")

HSS_OK = 0
ERRORS = {-1: "HSS_ERR_INVALID", -2: "HSS_ERR_WORKSPACE", -3: "HSS_ERR_ROUND_LIMIT", -4: "HSS_ERR_TIMEOUT",
          -5: "HSS_ERR_CUDA", -6: "HSS_ERR_CAPACITY", -7: "HSS_ERR_NOALLOC_LIMIT"}
ERR_INVALID, ERR_WORKSPACE, ERR_ROUND_LIMIT, ERR_TIMEOUT, ERR_CUDA, ERR_CAPACITY = -1, -2, -3, -4, -5, -6
KEY_TYPES = {"u64": 0, "i64": 1}
OP = {"sort": 0, "partition": 1, "local_sort": 2, "merge": 3, "exchange": 4, "sort_host": 5}
FLAG_SYNC = 1
FLAG_TIMING = 2
FLAG_HIST_PROBE = 4   # force the probe-side histogram
FLAG_HIST_STAGED = 8  # force the staged histogram in rounds whose probes share one interval
FLAG_HOST_ROUNDS = 16  # drive the splitter rounds from the host
FLAG_DEVICE_ROUNDS = 32  # always run the splitter rounds as the device-driven graph (default: from a shape's 2nd call) loop
MAX_ROUNDS = 64
NUM_PHASES = 4
PHASES = ("local_sort", "rounds", "exchange", "merge")


class HSSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_lib_or_none_strerror(code)})")


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("seed", ctypes.c_uint64), ("p", ctypes.c_uint32),
                ("oversample", ctypes.c_float), ("max_rounds", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("schedule", ctypes.c_uint32), ("schedule_k", ctypes.c_uint32)]


SCHEDULES = {"proportional": 0, "theory": 1, "equal": 2}


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("status", ctypes.c_int32), ("tol", ctypes.c_uint64),
                ("sample_size", ctypes.c_uint64 * MAX_ROUNDS), ("gamma", ctypes.c_uint64 * MAX_ROUNDS),
                ("unresolved", ctypes.c_uint64 * (MAX_ROUNDS + 1)), ("ms_phase", ctypes.c_float * NUM_PHASES),
                ("ms_radix_pass_total", ctypes.c_float), ("radix_pass_launches", ctypes.c_uint32),
                ("radix_pass_keys", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()


def _lib_or_none_strerror(code):
    try:
        return load().hss_strerror(code).decode()
    except Exception:
        return "?"


def load():
    """Load libhss.so (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhss.so is missing at {LIB_PATH}: build it with paper_1803_01237_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        P, U64, U32, I32, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
        lib.hss_workspace_bytes.argtypes = [I32, U64, ctypes.POINTER(Params), U32, I32, I32]
        lib.hss_workspace_bytes.restype = SZ
        lib.hss_local_sort.argtypes = [P, P, I32, U64, U32, P, P, P, SZ, P]
        lib.hss_rank_cuts.argtypes = [P, I32, U64, U32, P, U32, P, P, P]
        lib.hss_partition.argtypes = [P, I32, U64, ctypes.POINTER(Params), P, P, P, SZ, ctypes.POINTER(Stats), P]
        lib.hss_exchange.argtypes = [P, P, U64, U32, P, P, P, P, P, SZ, P]
        lib.hss_merge.argtypes = [P, P, I32, U64, U32, P, P, P, P, SZ, P]
        lib.hss_sort.argtypes = [P, P, I32, U64, ctypes.POINTER(Params), P, P, P, P, P, SZ, ctypes.POINTER(Stats), P]
        lib.hss_sort_host.argtypes = [P, P, I32, U64, ctypes.POINTER(Params), P, P, P, P, P, SZ, ctypes.POINTER(Stats), P]
        lib.hss_partition_with_proposal.argtypes = [P, I32, U64, ctypes.POINTER(Params), P, U32, P, P, P, SZ,
                                                    ctypes.POINTER(Stats), P]
        lib.hss_sort_with_proposal.argtypes = [P, P, I32, U64, ctypes.POINTER(Params), P, U32, P, P, P, P, P, SZ,
                                               ctypes.POINTER(Stats), P]
        lib.hss_sample_words.argtypes = [U64, U32, U32, U32, U32, P, P]
        lib.hss_cdf_model_bytes.argtypes = []
        lib.hss_cdf_model_bytes.restype = SZ
        lib.hss_cdf_work_bytes.argtypes = [U32]
        lib.hss_cdf_work_bytes.restype = SZ
        lib.hss_cdf_init.argtypes = [P, U64, I32, I32, U64, U64, P]
        lib.hss_cdf_grad.argtypes = [P, P, P, U32, U64, P, P, P, SZ, P]
        lib.hss_cdf_train.argtypes = [P, P, P, U32, U64, U32, ctypes.c_float, P, P, SZ, P]
        lib.hss_cdf_eval.argtypes = [P, P, U32, P, P]
        lib.hss_cdf_propose.argtypes = [P, U32, U32, ctypes.c_double, P, P]
        lib.hss_cdf_set_weights.argtypes = [P, I32, P]
        for name in ("hss_cdf_init", "hss_cdf_grad", "hss_cdf_train", "hss_cdf_eval", "hss_cdf_propose",
                     "hss_cdf_set_weights"):
            getattr(lib, name).restype = I32
        lib.hss_kernel_launch_count.argtypes = []
        lib.hss_kernel_launch_count.restype = U64
        lib.hss_strerror.argtypes = [I32]
        lib.hss_strerror.restype = ctypes.c_char_p
        for name in ("hss_local_sort", "hss_rank_cuts", "hss_partition", "hss_exchange", "hss_merge", "hss_sort",
                     "hss_sort_host", "hss_sample_words", "hss_partition_with_proposal", "hss_sort_with_proposal"):
            getattr(lib, name).restype = I32
        _lib = lib
        return lib


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _ptr(t):
    """Address for the C library: numpy arrays are host buffers (the host
    entry point); torch tensors must live in device memory."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    if not t.is_cuda:
        raise ValueError("device entry points take CUDA tensors (host arrays go through sort_host)")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc: int, where: str, allow=()):
    if rc != HSS_OK and rc not in allow:
        raise HSSError(rc, where)
    return rc


def _as_key_tensor(keys) -> torch.Tensor:
    if not isinstance(keys, torch.Tensor):
        raise TypeError("keys must be a CUDA int64 tensor (host arrays go through sort_host)")
    if keys.dtype not in (torch.int64,):
        raise TypeError("keys must be int64 tensors (u64 keys are passed by bit pattern)")
    if not keys.is_cuda:
        raise ValueError("keys must live in device memory (host arrays go through sort_host)")
    return keys.contiguous()


_ws_cache: dict = {}


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A cached device byte buffer of at least nbytes (grown on demand)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    buf = _ws_cache.get(dev)
    if buf is None or buf.numel() < nbytes:
        _ws_cache.pop(dev, None)
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        _ws_cache[dev] = buf
    return buf


def workspace_bytes(op: str, N: int, p: int, key_type: str = "u64", payload: bool = False,
                    oversample: float = 5.0, eps: float = 0.05) -> int:
    prm = Params(eps=eps, seed=0, p=p, oversample=oversample, max_rounds=0, flags=0)
    return int(load().hss_workspace_bytes(OP[op], N, ctypes.byref(prm), p, KEY_TYPES[key_type], int(payload)))


def cuts_to_numpy(raw: torch.Tensor):
    """Unpack an (n, 2) int64 tensor of hss_cut records into (key, seg, spos)."""
    a = raw.detach().cpu().numpy().reshape(-1, 2)
    key = a[:, 0].copy()
    seg = (a[:, 1] & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    spos = ((a[:, 1] >> 32) & 0xFFFFFFFF).astype(np.uint32)
    return key, seg, spos


def cuts_from_numpy(key, seg, spos, device) -> torch.Tensor:
    key = np.asarray(key).astype(np.uint64).view(np.int64)
    lo = np.asarray(seg, dtype=np.int32).view(np.uint32).astype(np.int64)
    hi = np.asarray(spos, dtype=np.uint32).astype(np.int64)
    packed = (lo | (hi << 32)).astype(np.int64)
    return torch.from_numpy(np.stack([key, packed], axis=1).copy()).to(device)


@dataclass
class Result:
    keys: torch.Tensor | None
    payload: torch.Tensor | None
    splitters: torch.Tensor        # (p-1, 2) int64: packed hss_cut records
    offsets: torch.Tensor          # (p+1,) int64
    rounds: int
    status: int
    tol: int
    sample_size: list = field(default_factory=list)
    gamma: list = field(default_factory=list)
    unresolved: list = field(default_factory=list)
    ms_phase: dict = field(default_factory=dict)
    ms_radix_pass_total: float = 0.0
    radix_pass_launches: int = 0
    radix_pass_keys: int = 0
    kernel_launches: int = 0

    def splitter_tags(self):
        return cuts_to_numpy(self.splitters)


def _result(keys, pay, spl, off, st: Stats) -> Result:
    R = st.rounds
    return Result(keys=keys, payload=pay, splitters=spl, offsets=off, rounds=R, status=st.status, tol=st.tol,
                  sample_size=[int(x) for x in st.sample_size[:R]], gamma=[int(x) for x in st.gamma[:R]],
                  unresolved=[int(x) for x in st.unresolved[:R + 1]],
                  ms_phase={PHASES[i]: float(st.ms_phase[i]) for i in range(NUM_PHASES)},
                  ms_radix_pass_total=float(st.ms_radix_pass_total), radix_pass_launches=int(st.radix_pass_launches),
                  radix_pass_keys=int(st.radix_pass_keys),
                  kernel_launches=int(st.kernel_launches))


def _params(p, eps, seed, oversample, max_rounds, flags, schedule="proportional", schedule_k=0):
    return Params(eps=float(eps), seed=int(seed) & ((1 << 64) - 1), p=int(p), oversample=float(oversample),
                  max_rounds=int(max_rounds), flags=int(flags), schedule=SCHEDULES[schedule],
                  schedule_k=int(schedule_k))


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def local_sort(keys, p: int, payload=None, key_type: str = "u64", out=None, out_payload=None, stream=None):
    """Stable sort of each of the p contiguous segments (hss_local_sort)."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    if out is None:
        out = torch.empty_like(keys)
    if payload is not None and out_payload is None:
        out_payload = torch.empty_like(payload)
    ws = workspace(workspace_bytes("local_sort", N, p, key_type, payload is not None), keys.device)
    rc = lib.hss_local_sort(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], N, p, _ptr(out), _ptr(out_payload),
                            _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "hss_local_sort")
    return (out, out_payload) if payload is not None else out


def rank_cuts(sorted_keys, p: int, cuts: torch.Tensor, key_type: str = "u64", want_seg_pos: bool = False, stream=None):
    """Global ranks (and optionally per-segment counts) of cuts (hss_rank_cuts)."""
    lib = load()
    sorted_keys = _as_key_tensor(sorted_keys)
    n = cuts.shape[0]
    ranks = torch.empty(n, dtype=torch.int64, device=sorted_keys.device)
    seg_pos = torch.empty((p, n), dtype=torch.int32, device=sorted_keys.device) if want_seg_pos else None
    rc = lib.hss_rank_cuts(_ptr(sorted_keys), KEY_TYPES[key_type], sorted_keys.numel(), p, _ptr(cuts.contiguous()), n,
                           _ptr(ranks), _ptr(seg_pos), _stream(stream))
    _check(rc, "hss_rank_cuts")
    return (ranks, seg_pos) if want_seg_pos else ranks


def partition(keys, p: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 0,
              key_type: str = "u64", flags: int = 0, stream=None, allow_round_limit: bool = False,
              schedule: str = "proportional", schedule_k: int = 0):
    """Splitters and bucket offsets (hss_partition).  Returns (Result, ws)
    where the first N*8 bytes of ws hold the locally sorted keys."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    prm = _params(p, eps, seed, oversample, max_rounds, flags, schedule, schedule_k)
    nb = int(lib.hss_workspace_bytes(OP["partition"], N, ctypes.byref(prm), p, KEY_TYPES[key_type], 0))
    ws = workspace(nb, keys.device)
    spl = torch.empty((max(p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    st = Stats()
    rc = lib.hss_partition(_ptr(keys), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(spl), _ptr(off), _ptr(ws),
                           ws.numel(), ctypes.byref(st), _stream(stream))
    _check(rc, "hss_partition", allow=(-3,) if allow_round_limit else ())
    return _result(None, None, spl[:p - 1], off, st), ws


def partition_async(keys, p: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 0,
                    key_type: str = "u64", flags: int = 0, stream=None):
    """hss_partition without statistics: returns (splitters, offsets, ws)
    without waiting for the GPU (the rounds run as a device-driven graph);
    call_stats(...) with the same arguments reads the statistics later."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_workspace_bytes(OP["partition"], N, ctypes.byref(prm), p, KEY_TYPES[key_type], 0))
    ws = workspace(nb, keys.device)
    spl = torch.empty((max(p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    rc = lib.hss_partition(_ptr(keys), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(spl), _ptr(off), _ptr(ws),
                           ws.numel(), None, _stream(stream))
    _check(rc, "hss_partition")
    return spl[:p - 1], off, ws


def _bind_call_stats(lib):
    """Argument types of hss_call_stats (bound on first use)."""
    if not hasattr(lib, "_call_stats_bound"):
        P = ctypes.c_void_p
        lib.hss_call_stats.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(Params), ctypes.c_int,
                                       ctypes.c_int, P, ctypes.c_size_t, ctypes.POINTER(Stats), P]
        lib.hss_call_stats.restype = ctypes.c_int
        lib._call_stats_bound = True
    return lib


def call_stats(op: str, N: int, p: int, eps: float, seed: int, ws: torch.Tensor, oversample: float = 5.0,
               max_rounds: int = 0, key_type: str = "u64", payload: bool = False, flags: int = 0, stream=None):
    """hss_call_stats: (status, Stats) of the last call on workspace ws."""
    lib = _bind_call_stats(load())
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    st = Stats()
    rc = lib.hss_call_stats(OP[op], N, ctypes.byref(prm), KEY_TYPES[key_type], int(payload), _ptr(ws), ws.numel(),
                            ctypes.byref(st), _stream(stream))
    return rc, st


def _proposal_tensor(proposal, keys: torch.Tensor):
    if proposal is None:
        return None, 0
    prop = _as_key_tensor(proposal)
    if prop.device != keys.device:
        raise ValueError("the proposal must be on the keys' device")
    return prop, prop.numel()


def partition_with_proposal(keys, p: int, eps: float, seed: int, proposal, oversample: float = 5.0,
                            max_rounds: int = 0, key_type: str = "u64", flags: int = 0, stream=None,
                            allow_round_limit: bool = False):
    """hss_partition after ranking the proposed cuts (keys of the caller's
    type, one device tensor) before round 1.  Returns (Result, ws)."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    prop, nprop = _proposal_tensor(proposal, keys)
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_workspace_bytes(OP["partition"], N, ctypes.byref(prm), p, KEY_TYPES[key_type], 0))
    ws = workspace(nb, keys.device)
    spl = torch.empty((max(p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    st = Stats()
    rc = lib.hss_partition_with_proposal(_ptr(keys), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(prop), nprop,
                                         _ptr(spl), _ptr(off), _ptr(ws), ws.numel(), ctypes.byref(st), _stream(stream))
    _check(rc, "hss_partition_with_proposal", allow=(-3,) if allow_round_limit else ())
    return _result(None, None, spl[:p - 1], off, st), ws


def sort_with_proposal(keys, p: int, eps: float, seed: int, proposal, payload=None, oversample: float = 5.0,
                       max_rounds: int = 0, key_type: str = "u64", flags: int = 0, out=None, out_payload=None,
                       stream=None) -> "Result":
    """hss_sort after ranking the proposed cuts before round 1."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    prop, nprop = _proposal_tensor(proposal, keys)
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_workspace_bytes(OP["sort"], N, ctypes.byref(prm), p, KEY_TYPES[key_type], int(payload is not None)))
    ws = workspace(nb, keys.device)
    if out is None:
        out = torch.empty_like(keys)
    if payload is not None and out_payload is None:
        out_payload = torch.empty_like(payload)
    spl = torch.empty((max(p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    st = Stats()
    rc = lib.hss_sort_with_proposal(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(prop),
                                    nprop, _ptr(out), _ptr(out_payload), _ptr(spl), _ptr(off), _ptr(ws), ws.numel(),
                                    ctypes.byref(st), _stream(stream))
    _check(rc, "hss_sort_with_proposal")
    return _result(out, out_payload, spl[:p - 1], off, st)


def exchange(sorted_keys, p: int, seg_pos: torch.Tensor, offsets: torch.Tensor, sorted_payload=None, stream=None):
    """Runs of the locally sorted segments to their buckets (hss_exchange)."""
    lib = load()
    sorted_keys = _as_key_tensor(sorted_keys)
    N = sorted_keys.numel()
    bk = torch.empty_like(sorted_keys)
    bp = torch.empty_like(sorted_payload) if sorted_payload is not None else None
    ws = workspace(workspace_bytes("exchange", N, p), sorted_keys.device)
    rc = lib.hss_exchange(_ptr(sorted_keys), _ptr(sorted_payload), N, p, _ptr(seg_pos.contiguous()), _ptr(offsets),
                          _ptr(bk), _ptr(bp), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "hss_exchange")
    return (bk, bp) if sorted_payload is not None else bk


def merge(bucket_keys, p: int, offsets: torch.Tensor, bucket_payload=None, key_type: str = "u64", stream=None):
    """Stable merge of the runs inside each bucket (hss_merge)."""
    lib = load()
    bucket_keys = _as_key_tensor(bucket_keys)
    N = bucket_keys.numel()
    out = torch.empty_like(bucket_keys)
    outp = torch.empty_like(bucket_payload) if bucket_payload is not None else None
    ws = workspace(workspace_bytes("merge", N, p, key_type, bucket_payload is not None), bucket_keys.device)
    rc = lib.hss_merge(_ptr(bucket_keys), _ptr(bucket_payload), KEY_TYPES[key_type], N, p, _ptr(offsets), _ptr(out),
                       _ptr(outp), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "hss_merge")
    return (out, outp) if bucket_payload is not None else out


def sort(keys, p: int, eps: float, seed: int, payload=None, oversample: float = 5.0, max_rounds: int = 0,
         key_type: str = "u64", flags: int = 0, out=None, out_payload=None, stream=None,
         schedule: str = "proportional", schedule_k: int = 0) -> Result:
    """The whole method (hss_sort): globally sorted keys, splitters, offsets."""
    lib = load()
    keys = _as_key_tensor(keys)
    N = keys.numel()
    prm = _params(p, eps, seed, oversample, max_rounds, flags, schedule, schedule_k)
    nb = int(lib.hss_workspace_bytes(OP["sort"], N, ctypes.byref(prm), p, KEY_TYPES[key_type], int(payload is not None)))
    ws = workspace(nb, keys.device)
    if out is None:
        out = torch.empty_like(keys)
    if payload is not None and out_payload is None:
        out_payload = torch.empty_like(payload)
    spl = torch.empty((max(p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    st = Stats()
    rc = lib.hss_sort(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(out), _ptr(out_payload),
                      _ptr(spl), _ptr(off), _ptr(ws), ws.numel(), ctypes.byref(st), _stream(stream))
    _check(rc, "hss_sort")
    return _result(out, out_payload, spl[:p - 1], off, st)


def sort_host(keys: np.ndarray, p: int, eps: float, seed: int, payload: np.ndarray | None = None,
              oversample: float = 5.0, max_rounds: int = 0, key_type: str = "u64", flags: int = 0,
              out: np.ndarray | None = None, out_payload: np.ndarray | None = None, stream=None):
    """hss_sort_host: host arrays in, host arrays out (copies inside the call)."""
    lib = load()
    keys = np.ascontiguousarray(keys)
    N = keys.shape[0]
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_workspace_bytes(OP["sort_host"], N, ctypes.byref(prm), p, KEY_TYPES[key_type],
                                     int(payload is not None)))
    ws = workspace(nb)
    if out is None:
        out = np.empty_like(keys)
    if payload is not None and out_payload is None:
        out_payload = np.empty_like(payload)
    spl = np.empty((max(p - 1, 1), 2), dtype=np.int64)
    off = np.empty(p + 1, dtype=np.uint64)
    st = Stats()
    rc = lib.hss_sort_host(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], N, ctypes.byref(prm), _ptr(out),
                           _ptr(out_payload), _ptr(spl), _ptr(off), _ptr(ws), ws.numel(), ctypes.byref(st),
                           _stream(stream))
    _check(rc, "hss_sort_host")
    return out, out_payload, spl[:p - 1], off, st


def sample_words(seed: int, seg: int, rnd: int, spos0: int, count: int, device="cuda", stream=None) -> torch.Tensor:
    """The Philox words of positions spos0.. of segment seg in round rnd."""
    lib = load()
    out = torch.empty(count, dtype=torch.int64, device=device)
    rc = lib.hss_sample_words(int(seed) & ((1 << 64) - 1), seg, rnd, spos0, count, _ptr(out), _stream(stream))
    _check(rc, "hss_sample_words")
    return out


class Tuning(ctypes.Structure):
    _fields_ = [("chip_max_keys", ctypes.c_uint32), ("child_interp", ctypes.c_uint32),
                ("child_bucket_keys", ctypes.c_uint32), ("pack_keys", ctypes.c_uint32),
                ("first_split", ctypes.c_uint32), ("split_scatter", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]


def set_tuning(chip_max_keys: int = 0, child_interp: int = 0, child_bucket_keys: int = 0, pack_keys: int = 0,
               first_split: int = 0, split_scatter: int = 0):
    """hss_set_tuning: process-wide choices of the segmented sort (results unchanged)."""
    lib = load()
    t = Tuning(chip_max_keys=int(chip_max_keys), child_interp=int(child_interp),
               child_bucket_keys=int(child_bucket_keys), pack_keys=int(pack_keys), first_split=int(first_split),
               split_scatter=int(split_scatter))
    _check(lib.hss_set_tuning(ctypes.byref(t)), "hss_set_tuning")


def reset_tuning():
    _check(load().hss_set_tuning(None), "hss_set_tuning")


def get_tuning() -> dict:
    t = Tuning()
    _check(load().hss_get_tuning(ctypes.byref(t)), "hss_get_tuning")
    return {"chip_max_keys": t.chip_max_keys, "child_interp": t.child_interp,
            "child_bucket_keys": t.child_bucket_keys, "pack_keys": t.pack_keys, "first_split": t.first_split,
            "split_scatter": t.split_scatter}


def launch_count() -> int:
    return int(load().hss_kernel_launch_count())


def strerror(code: int) -> str:
    return load().hss_strerror(code).decode()


# ---------------------------------------------------------------------------
# Learned splitter proposal: the 1-32-32-1 CDF network (hss_cdf_*)
# ---------------------------------------------------------------------------
CDF_NPARAM = 1153
CDF_FEATURES = {"linear": 0, "log": 1}
CDF_WEIGHTS = {"fp32": 0, "bf16": 1}


class CDFModel:
    """A device-resident CDF network (one hss_cdf_model struct in a uint8
    tensor).  theta/m/v views alias the struct's float arrays."""

    def __init__(self, device=None):
        lib = load()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nbytes = int(lib.hss_cdf_model_bytes())
        self.buf = torch.zeros(self.nbytes, dtype=torch.uint8, device=dev)
        self._work = torch.empty(0, dtype=torch.uint8, device=dev)
        self.key_type = "u64"

    @property
    def theta(self) -> torch.Tensor:
        return self.buf[:4 * CDF_NPARAM].view(torch.float32)

    @property
    def step(self) -> int:
        return int(self.buf[12 * CDF_NPARAM:12 * CDF_NPARAM + 4].view(torch.int32).item())

    def init(self, seed: int, feature: str, lo_key: int, hi_key: int, key_type: str = "u64", stream=None):
        self.key_type = key_type
        rc = load().hss_cdf_init(_ptr(self.buf), seed & ((1 << 64) - 1), CDF_FEATURES[feature], KEY_TYPES[key_type],
                                 lo_key & ((1 << 64) - 1), hi_key & ((1 << 64) - 1), _stream(stream))
        _check(rc, "hss_cdf_init")
        return self

    def set_weights(self, weights: str, stream=None):
        """"fp32", or "bf16": later evaluations use the parameters rounded to
        bfloat16 (hss_cdf_set_weights)."""
        rc = load().hss_cdf_set_weights(_ptr(self.buf), CDF_WEIGHTS[weights], _stream(stream))
        _check(rc, "hss_cdf_set_weights")
        return self

    def _ws(self, n: int) -> torch.Tensor:
        nb = int(load().hss_cdf_work_bytes(n))
        if self._work.numel() < nb:
            self._work = torch.empty(nb, dtype=torch.uint8, device=self.buf.device)
        return self._work

    def grad(self, keys, ranks, N: int, stream=None):
        """(gradient[1153], loss) at the current parameters."""
        keys = _as_key_tensor(keys)
        ranks = ranks.contiguous()
        n = keys.numel()
        g = torch.empty(CDF_NPARAM, dtype=torch.float32, device=self.buf.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.buf.device)
        ws = self._ws(n)
        rc = load().hss_cdf_grad(_ptr(self.buf), _ptr(keys), _ptr(ranks), n, N, _ptr(g), _ptr(loss), _ptr(ws),
                                 ws.numel(), _stream(stream))
        _check(rc, "hss_cdf_grad")
        return g, loss

    def train(self, keys, ranks, N: int, steps: int, lr: float = 0.01, stream=None) -> torch.Tensor:
        keys = _as_key_tensor(keys)
        ranks = ranks.contiguous()
        n = keys.numel()
        loss = torch.empty(1, dtype=torch.float32, device=self.buf.device)
        ws = self._ws(n)
        rc = load().hss_cdf_train(_ptr(self.buf), _ptr(keys), _ptr(ranks), n, N, steps, float(lr), _ptr(loss),
                                  _ptr(ws), ws.numel(), _stream(stream))
        _check(rc, "hss_cdf_train")
        return loss

    def eval(self, keys, stream=None) -> torch.Tensor:
        keys = _as_key_tensor(keys)
        y = torch.empty(keys.numel(), dtype=torch.float32, device=self.buf.device)
        rc = load().hss_cdf_eval(_ptr(self.buf), _ptr(keys), keys.numel(), _ptr(y), _stream(stream))
        _check(rc, "hss_cdf_eval")
        return y

    def propose(self, p: int, per_splitter: int = 1, delta: float = 0.0, stream=None) -> torch.Tensor:
        out = torch.empty(max(p - 1, 0) * per_splitter, dtype=torch.int64, device=self.buf.device)
        rc = load().hss_cdf_propose(_ptr(self.buf), p, per_splitter, float(delta), _ptr(out), _stream(stream))
        _check(rc, "hss_cdf_propose")
        return out


def training_pairs(res: "Result"):
    """(keys, ranks) training points of the CDF network from an HSS result:
    every final splitter that is an input key or a proposed cut, with its
    exact rank chi(i) (offsets[i+1]).  Sentinel splitters are dropped."""
    spl = res.splitters
    seg = (spl[:, 1] & 0xFFFFFFFF).to(torch.int32)
    keep = seg >= -1
    return spl[:, 0][keep].contiguous(), res.offsets[1:-1][keep].contiguous()


# ---------------------------------------------------------------------------
# Batches of independent jobs (hss_sort_batch / hss_partition_batch)
# ---------------------------------------------------------------------------
class JobStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint32), ("status", ctypes.c_int32), ("tol", ctypes.c_uint64),
                ("sample_size", ctypes.c_uint64 * MAX_ROUNDS), ("gamma", ctypes.c_uint64 * MAX_ROUNDS),
                ("unresolved", ctypes.c_uint64 * (MAX_ROUNDS + 1))]


class BatchStats(ctypes.Structure):
    _fields_ = [("njobs", ctypes.c_uint32), ("max_rounds", ctypes.c_uint32), ("lockstep_rounds", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("total_samples", ctypes.c_uint64), ("total_keys", ctypes.c_uint64),
                ("total_segments", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("ms_phase", ctypes.c_float * NUM_PHASES)]


@dataclass
class BatchResult:
    keys: torch.Tensor | None
    payload: torch.Tensor | None
    splitters: torch.Tensor      # (sum (p_j - 1), 2) packed hss_cut records, job-major
    offsets: torch.Tensor        # (sum (p_j + 1),) job-relative offsets, job-major
    sizes: list
    ps: list
    status: int
    job_rounds: list
    job_sample_size: list
    job_gamma: list
    job_unresolved: list
    job_status: list
    job_tol: list
    lockstep_rounds: int
    total_samples: int
    kernel_launches: int
    ms_phase: dict

    def job_offsets(self, j: int) -> torch.Tensor:
        o = sum(p + 1 for p in self.ps[:j])
        return self.offsets[o:o + self.ps[j] + 1]

    def job_splitters(self, j: int) -> torch.Tensor:
        o = sum(p - 1 for p in self.ps[:j])
        return self.splitters[o:o + self.ps[j] - 1]


def _bind_batch(lib):
    """Argument types of the batched entry points (bound on first use)."""
    if not hasattr(lib, "_batch_bound"):
        P, U64, U32, I32, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
        lib.hss_batch_workspace_bytes.argtypes = [P, P, U32, ctypes.POINTER(Params), I32, I32, I32]
        lib.hss_batch_workspace_bytes.restype = SZ
        lib.hss_sort_batch.argtypes = [P, P, I32, P, P, U32, ctypes.POINTER(Params), P, P, P, P, P, SZ,
                                       ctypes.POINTER(BatchStats), P, P]
        lib.hss_sort_batch.restype = I32
        lib.hss_partition_batch.argtypes = [P, I32, P, P, U32, ctypes.POINTER(Params), P, P, P, SZ,
                                            ctypes.POINTER(BatchStats), P, P]
        lib.hss_partition_batch.restype = I32
        lib.hss_sort_batch_seeded.argtypes = [P, P, I32, P, P, P, U32, ctypes.POINTER(Params), P, P, P, P, P, SZ,
                                              ctypes.POINTER(BatchStats), P, P]
        lib.hss_sort_batch_seeded.restype = I32
        lib.hss_partition_batch_seeded.argtypes = [P, I32, P, P, P, U32, ctypes.POINTER(Params), P, P, P, SZ,
                                                   ctypes.POINTER(BatchStats), P, P]
        lib.hss_partition_batch_seeded.restype = I32
        lib._batch_bound = True
    return lib


def _batch(keys, sizes, ps, eps, seed, payload, oversample, max_rounds, key_type, flags, sort, out, out_payload,
           stream, seeds=None, ws=None):
    lib = _bind_batch(load())
    keys = _as_key_tensor(keys)
    sizes = np.ascontiguousarray(np.asarray(sizes, dtype=np.uint64))
    ps = np.ascontiguousarray(np.asarray(ps, dtype=np.uint32))
    nj = int(sizes.shape[0])
    if int(sizes.sum()) != keys.numel():
        raise ValueError("the job sizes must add up to the number of keys")
    prm = _params(1, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_batch_workspace_bytes(_ptr(sizes), _ptr(ps), nj, ctypes.byref(prm), KEY_TYPES[key_type],
                                           int(payload is not None), int(sort)))
    if nb == 0:
        raise HSSError(ERR_INVALID, "hss_batch_workspace_bytes")
    if ws is None or ws.numel() < nb:
        ws = workspace(nb, keys.device)
    sd = None
    if seeds is not None:
        sd = np.ascontiguousarray(np.asarray([int(x) & ((1 << 64) - 1) for x in seeds], dtype=np.uint64))
        if sd.shape[0] != nj:
            raise ValueError("one seed per job")
    S_tot = int((ps.astype(np.int64) - 1).sum())
    O_tot = int((ps.astype(np.int64) + 1).sum())
    spl = torch.empty((max(S_tot, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(O_tot, dtype=torch.int64, device=keys.device)
    st = BatchStats()
    js = (JobStats * nj)()
    if sort:
        if out is None:
            out = torch.empty_like(keys)
        if payload is not None and out_payload is None:
            out_payload = torch.empty_like(payload)
        rc = lib.hss_sort_batch_seeded(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], _ptr(sizes), _ptr(ps),
                                       _ptr(sd), nj, ctypes.byref(prm), _ptr(out), _ptr(out_payload), _ptr(spl),
                                       _ptr(off), _ptr(ws), ws.numel(), ctypes.byref(st), js, _stream(stream))
    else:
        rc = lib.hss_partition_batch_seeded(_ptr(keys), KEY_TYPES[key_type], _ptr(sizes), _ptr(ps), _ptr(sd), nj,
                                            ctypes.byref(prm), _ptr(spl), _ptr(off), _ptr(ws), ws.numel(),
                                            ctypes.byref(st), js, _stream(stream))
    if rc in (ERR_INVALID, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT):
        raise HSSError(rc, "hss_sort_batch" if sort else "hss_partition_batch")
    return BatchResult(
        keys=out if sort else None, payload=out_payload if sort else None, splitters=spl[:S_tot], offsets=off,
        sizes=[int(x) for x in sizes], ps=[int(x) for x in ps], status=rc,
        job_rounds=[int(x.rounds) for x in js], job_status=[int(x.status) for x in js],
        job_tol=[int(x.tol) for x in js],
        job_sample_size=[[int(v) for v in x.sample_size[:x.rounds]] for x in js],
        job_gamma=[[int(v) for v in x.gamma[:x.rounds]] for x in js],
        job_unresolved=[[int(v) for v in x.unresolved[:x.rounds + 1]] for x in js],
        lockstep_rounds=int(st.lockstep_rounds), total_samples=int(st.total_samples),
        kernel_launches=int(st.kernel_launches),
        ms_phase={PHASES[i]: float(st.ms_phase[i]) for i in range(NUM_PHASES)})


def batch_workspace_bytes(sizes, ps, eps: float, sort: bool = True, payload: bool = False, key_type: str = "u64",
                          oversample: float = 5.0) -> int:
    """hss_batch_workspace_bytes of a job list (0 when the list is refused)."""
    lib = load()
    P, U32, I32, SZ = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
    lib.hss_batch_workspace_bytes.argtypes = [P, P, U32, ctypes.POINTER(Params), I32, I32, I32]
    lib.hss_batch_workspace_bytes.restype = SZ
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.uint64))
    pp = np.ascontiguousarray(np.asarray(ps, dtype=np.uint32))
    prm = _params(1, eps, 0, oversample, 0, 0)
    return int(lib.hss_batch_workspace_bytes(_ptr(sz), _ptr(pp), int(sz.shape[0]), ctypes.byref(prm),
                                             KEY_TYPES[key_type], int(payload), int(sort)))


def sort_batch(keys, sizes, ps, eps: float, seed: int, payload=None, oversample: float = 5.0, max_rounds: int = 0,
               key_type: str = "u64", flags: int = 0, out=None, out_payload=None, stream=None,
               seeds=None) -> BatchResult:
    """hss_sort of every job of a batch (job j: the next sizes[j] keys, ps[j]
    processors, seed + j, or seeds[j] when seeds is given), all jobs
    together."""
    return _batch(keys, sizes, ps, eps, seed, payload, oversample, max_rounds, key_type, flags, True, out,
                  out_payload, stream, seeds)


def partition_batch(keys, sizes, ps, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 0,
                    key_type: str = "u64", flags: int = 0, stream=None, seeds=None, ws=None) -> BatchResult:
    """hss_partition of every job of a batch, all jobs together (seeds as
    for sort_batch; ws: a workspace to use when large enough)."""
    return _batch(keys, sizes, ps, eps, seed, None, oversample, max_rounds, key_type, flags, False, None, None, stream,
                  seeds, ws)


# ---------------------------------------------------------------------------
# Two-stage HSS (hss_sort_two_stage)
# ---------------------------------------------------------------------------
class TwoStageStats(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_uint32), ("status", ctypes.c_int32), ("kernel_launches", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("stage1", Stats), ("stage2", BatchStats)]


@dataclass
class TwoStageResult:
    keys: torch.Tensor
    payload: torch.Tensor | None
    offsets: torch.Tensor          # (p + 1,) absolute bucket offsets
    group_splitters: torch.Tensor  # (r - 1, 2) packed hss_cut records (stage 1)
    splitters: torch.Tensor        # (r (p/r - 1), 2) packed hss_cut records (stage 2, group-major)
    groups: int
    status: int
    stage1: Result                 # the group split (keys None; offsets = group offsets)
    group_rounds: list
    group_sample_size: list
    group_gamma: list
    group_unresolved: list
    group_status: list
    group_tol: list
    lockstep_rounds: int
    kernel_launches: int
    ms_phase: dict                 # stage-1 and stage-2 phases

    def group_splitters_of(self, g: int) -> torch.Tensor:
        pg = (self.offsets.numel() - 1) // self.groups
        return self.splitters[g * (pg - 1):(g + 1) * (pg - 1)]


def _bind_two_stage(lib):
    """Argument types of the two-stage entry points (bound on first use)."""
    if not hasattr(lib, "_two_stage_bound"):
        P, U64, U32, I32, SZ = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
        lib.hss_two_stage_workspace_bytes.argtypes = [U64, ctypes.POINTER(Params), U32, I32, I32]
        lib.hss_two_stage_workspace_bytes.restype = SZ
        lib.hss_sort_two_stage.argtypes = [P, P, I32, U64, ctypes.POINTER(Params), U32, P, P, P, P, P, P, SZ,
                                           ctypes.POINTER(TwoStageStats), P, P]
        lib.hss_sort_two_stage.restype = I32
        lib._two_stage_bound = True
    return lib


def sort_two_stage(keys, p: int, groups: int, eps: float, seed: int, payload=None, oversample: float = 5.0,
                   max_rounds: int = 0, key_type: str = "u64", flags: int = 0, out=None, out_payload=None,
                   stream=None) -> TwoStageResult:
    """Two-stage HSS (hss_sort_two_stage): the p processors' keys split into
    `groups` groups, then each group sorted over its p / groups processors
    with seed + 1 + g."""
    lib = _bind_two_stage(load())
    keys = _as_key_tensor(keys)
    N = keys.numel()
    r = int(groups)
    prm = _params(p, eps, seed, oversample, max_rounds, flags)
    nb = int(lib.hss_two_stage_workspace_bytes(N, ctypes.byref(prm), r, KEY_TYPES[key_type], int(payload is not None)))
    if nb == 0:
        raise HSSError(ERR_INVALID, "hss_two_stage_workspace_bytes")
    ws = workspace(nb, keys.device)
    if out is None:
        out = torch.empty_like(keys)
    if payload is not None and out_payload is None:
        out_payload = torch.empty_like(payload)
    pg = p // r
    gspl = torch.empty((max(r - 1, 1), 2), dtype=torch.int64, device=keys.device)
    spl = torch.empty((max(r * (pg - 1), 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(p + 1, dtype=torch.int64, device=keys.device)
    st = TwoStageStats()
    js = (JobStats * r)()
    rc = lib.hss_sort_two_stage(_ptr(keys), _ptr(payload), KEY_TYPES[key_type], N, ctypes.byref(prm), r, _ptr(out),
                                _ptr(out_payload), _ptr(gspl), _ptr(spl), _ptr(off), _ptr(ws), ws.numel(),
                                ctypes.byref(st), js, _stream(stream))
    if rc in (ERR_INVALID, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT):
        raise HSSError(rc, "hss_sort_two_stage")
    goff = off[::pg].clone()
    s1 = _result(None, None, gspl[:r - 1], goff, st.stage1)
    ms = {f"stage1_{PHASES[i]}": float(st.stage1.ms_phase[i]) for i in range(3)}
    ms.update({f"stage2_{PHASES[i]}": float(st.stage2.ms_phase[i]) for i in range(NUM_PHASES)})
    return TwoStageResult(
        keys=out, payload=out_payload, offsets=off, group_splitters=gspl[:r - 1], splitters=spl[:r * (pg - 1)],
        groups=r, status=rc, stage1=s1,
        group_rounds=[int(x.rounds) for x in js], group_status=[int(x.status) for x in js],
        group_tol=[int(x.tol) for x in js],
        group_sample_size=[[int(v) for v in x.sample_size[:x.rounds]] for x in js],
        group_gamma=[[int(v) for v in x.gamma[:x.rounds]] for x in js],
        group_unresolved=[[int(v) for v in x.unresolved[:x.rounds + 1]] for x in js],
        lockstep_rounds=int(st.stage2.lockstep_rounds), kernel_launches=int(st.kernel_launches), ms_phase=ms)
