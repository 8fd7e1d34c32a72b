"""CPU oracle for Histogram Sort with Sampling (Harsh, Kale, Solomonik, SPAA'19).

TEST INFRASTRUCTURE ONLY.  A plain single-threaded C restatement of the method
(hss_oracle.c) behind a small numpy wrapper.  Beside it, cpu_baselines.cpp
holds the benchmark's timed CPU references (HSS on all cores with OpenMP, and
std::sort); they are checked against the oracle, never the other way round.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import this package; the
product library never links or calls it, and the two share no code.

Functions cite the paper's sections:
  philox4x32_10      - the counter-based generator (Salmon et al., SC'11)
  sample_draw        - the per-key Bernoulli word of Sec. 4.2.1 / Sec. 6
  segment_sort       - the local sort with implicit tagging (Sec. 6.1)
  cut_rank           - the histogram of one probe (Sec. 3.3 step 2)
  hss                - the whole method: rounds of Sec. 4.2.2, exchange and
                       merge of Sec. 3.1 step 3
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hss_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_ROUNDS = 64


_BASE_SRC = os.path.join(_HERE, "cpu_baselines.cpp")
_BASE_PATH = os.path.join(_OUT_DIR, "libcpu_baselines.so")
_base = None


def build_baselines(force: bool = False) -> str:
    """Compile the timed CPU baselines (OpenMP HSS, std::sort) with g++."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_BASE_PATH)
            and os.path.getmtime(_BASE_PATH) >= os.path.getmtime(_BASE_SRC)):
        return _BASE_PATH
    tmp = _BASE_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-std=c++17", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _BASE_SRC])
    os.replace(tmp, _BASE_PATH)
    return _BASE_PATH


def _load_baselines():
    global _base
    with _lock:
        if _base is None:
            lib = ctypes.CDLL(build_baselines())
            P = ctypes.c_void_p
            lib.cpu_baseline_threads.restype = ctypes.c_int
            lib.cpu_std_sort.argtypes = [P, ctypes.c_uint64]
            lib.cpu_std_sort.restype = None
            lib.cpu_hss_omp.argtypes = [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_float, ctypes.c_uint32, P, P, P, P, P, P, P]
            lib.cpu_hss_omp.restype = ctypes.c_int
            _base = lib
    return _base


def baseline_threads() -> int:
    """Threads the OpenMP baseline uses (OMP_NUM_THREADS or all host cores)."""
    return int(_load_baselines().cpu_baseline_threads())


def std_sort(keys) -> np.ndarray:
    """std::sort of u64 keys on one core (a timed reference, not the oracle)."""
    out = np.array(keys, dtype=np.uint64, copy=True)
    _load_baselines().cpu_std_sort(_ptr(out), out.shape[0])
    return out


def hss_omp(keys, p: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 64, sort: bool = True):
    """HSS on all host cores (OpenMP), u64 keys alone: the same steps and
    readings as ``hss``, run in parallel (a timed baseline, not the oracle).
    Returns (splitter_key, splitter_seg, splitter_spos, offsets, out_keys,
    rounds, sample_size, status)."""
    lib = _load_baselines()
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    N, S = k.shape[0], max(p - 1, 0)
    sk = np.zeros(max(S, 1), dtype=np.uint64)
    ss = np.zeros(max(S, 1), dtype=np.int32)
    sp = np.zeros(max(S, 1), dtype=np.uint32)
    off = np.zeros(p + 1, dtype=np.uint64)
    out = np.empty(max(N, 1), dtype=np.uint64) if sort else None
    rounds = ctypes.c_uint32(0)
    z = np.zeros(64, dtype=np.uint64)
    rc = lib.cpu_hss_omp(_ptr(k), N, p, float(eps), int(seed) & ((1 << 64) - 1), float(oversample), max_rounds,
                         _ptr(sk), _ptr(ss), _ptr(sp), _ptr(off), _ptr(out), ctypes.byref(rounds), _ptr(z))
    if rc == -1:
        raise ValueError("cpu_hss_omp: invalid arguments")
    R = int(rounds.value)
    return sk[:S], ss[:S], sp[:S], off, (out[:N] if sort else None), R, z[:R], rc


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no vector intrinsics)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_uint32),
        ("status", ctypes.c_int32),
        ("tol", ctypes.c_uint64),
        ("sample_size", ctypes.c_uint64 * MAX_ROUNDS),
        ("gamma", ctypes.c_uint64 * MAX_ROUNDS),
        ("unresolved", ctypes.c_uint64 * (MAX_ROUNDS + 1)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_sample_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_sample_draw.restype = ctypes.c_uint64
            lib.oracle_threshold.argtypes = [ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, P, P]
            lib.oracle_threshold.restype = None
            lib.oracle_tolerance.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double]
            lib.oracle_tolerance.restype = ctypes.c_uint64
            lib.oracle_segment_sort.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, P, P]
            lib.oracle_segment_sort.restype = None
            lib.oracle_cut_rank.argtypes = [P, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                            ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32]
            lib.oracle_cut_rank.restype = ctypes.c_uint64
            lib.oracle_hss.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_float, ctypes.c_uint32, P, ctypes.c_uint32,
                                       ctypes.c_int, ctypes.c_uint32,
                                       P, P, P, P, P, P, ctypes.POINTER(_Stats), P, P, P, P, ctypes.c_uint64]
            lib.oracle_hss.restype = ctypes.c_int
            lib.oracle_hss_groups.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_float,
                                              ctypes.c_uint32, P, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                              P, P, P, P, P, P, ctypes.POINTER(_Stats), P, P, P, P, ctypes.c_uint64]
            lib.oracle_hss_groups.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


KEY_U64 = 0
KEY_I64 = 1


def _keys_u64(keys):
    keys = np.ascontiguousarray(keys)
    if keys.dtype == np.int64:
        return keys.view(np.uint64), KEY_I64
    if keys.dtype != np.uint64:
        raise TypeError(f"keys must be uint64 or int64, got {keys.dtype}")
    return keys, KEY_U64


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11): 4 x u32 -> 4 x u32."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample_draw(seed: int, seg: int, spos: int, rnd: int) -> int:
    """64-bit Bernoulli word of the key at (seg, spos) in round rnd."""
    return int(_load().oracle_sample_draw(seed, seg, spos, rnd))


def threshold(oversample: float, p: int, gamma: int):
    """(T, take_all) for q = min(1, s*p/|gamma|)."""
    lib = _load()
    T = ctypes.c_uint64(0)
    ta = ctypes.c_int(0)
    lib.oracle_threshold(float(np.float32(oversample)), p, gamma, ctypes.byref(T), ctypes.byref(ta))
    return int(T.value), bool(ta.value)


def tolerance(N: int, p: int, eps: float) -> int:
    """tol = floor(N*eps/(2p)), the half-width of the target range (Sec. 2)."""
    return int(_load().oracle_tolerance(N, p, eps))


def segment_bounds(N: int, p: int) -> np.ndarray:
    return np.array([(s * N) // p for s in range(p + 1)], dtype=np.uint64)


def segment_sort(keys, p: int, payload=None):
    """Stable local sort of every processor's contiguous segment (Sec. 5, 6.1)."""
    lib = _load()
    k, kt = _keys_u64(keys)
    N = k.shape[0]
    out = np.empty(N, dtype=np.uint64)
    pay = None if payload is None else np.ascontiguousarray(payload, dtype=np.uint32)
    opay = None if payload is None else np.empty(N, dtype=np.uint32)
    lib.oracle_segment_sort(_ptr(k), _ptr(pay), N, kt, p, _ptr(out), _ptr(opay))
    if kt == KEY_I64:
        out = out.view(np.int64)
    return (out, opay) if payload is not None else out


def cut_rank(keys, p: int, key, seg: int = -1, spos: int = 0, member: bool = True) -> int:
    """Global rank (#keys strictly below) of a cut, summed over the locally
    sorted segments (the histogram of Sec. 3.3 step 2)."""
    lib = _load()
    k, kt = _keys_u64(keys)
    kind = 1 if member else 2
    kv = int(np.array([key]).astype(np.int64 if kt == KEY_I64 else np.uint64).view(np.uint64)[0])
    return int(lib.oracle_cut_rank(_ptr(k), k.shape[0], kt, p, kind, kv, seg, spos))


@dataclass
class HSSResult:
    splitter_key: np.ndarray
    splitter_seg: np.ndarray
    splitter_spos: np.ndarray
    offsets: np.ndarray
    rounds: int
    status: int
    tol: int
    sample_size: np.ndarray
    gamma: np.ndarray
    unresolved: np.ndarray
    out_keys: np.ndarray | None = None
    out_payload: np.ndarray | None = None
    trace_lrank: np.ndarray | None = None
    trace_urank: np.ndarray | None = None
    trace_resolved: np.ndarray | None = None
    samples: list = field(default_factory=list)


SCHEDULES = {"proportional": 0, "theory": 1, "equal": 2}


def hss(keys, p: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 64,
        payload=None, sort: bool = True, trace: bool = False, proposal=None, schedule: str = "proportional",
        schedule_k: int = 0) -> HSSResult:
    """Run the whole method (Sec. 4.2.2 rounds, then exchange and merge).

    schedule: "proportional" (s p / |gamma| per key, Sec. 6), "theory" (the
    k-round s_j = (2 ln p / eps)^(j/k) schedule of Theorem 4.7, k =
    schedule_k) or "equal" (s p / nint expected samples per distinct
    unresolved interval, the HykSort way of Sec. 4.2.2)."""
    lib = _load()
    k, kt = _keys_u64(keys)
    N = int(k.shape[0])
    S = max(p - 1, 0)
    spl_key = np.zeros(max(S, 1), dtype=np.uint64)
    spl_seg = np.zeros(max(S, 1), dtype=np.int32)
    spl_spos = np.zeros(max(S, 1), dtype=np.uint32)
    offsets = np.zeros(p + 1, dtype=np.uint64)
    pay = None if payload is None else np.ascontiguousarray(payload, dtype=np.uint32)
    out_keys = np.empty(max(N, 1), dtype=np.uint64) if sort else None
    out_pay = np.empty(max(N, 1), dtype=np.uint32) if (sort and payload is not None) else None
    st = _Stats()
    tl = tu = tr = ts = None
    cap = 0
    if trace:
        tl = np.zeros((max_rounds + 1) * max(S, 1), dtype=np.uint64)
        tu = np.zeros_like(tl)
        tr = np.zeros((max_rounds + 1) * max(S, 1), dtype=np.uint8)
        cap = 1 << 22
        ts = np.zeros(3 * cap, dtype=np.uint64)
    prop = None
    nprop = 0
    if proposal is not None:
        prop = np.ascontiguousarray(np.asarray(proposal).astype(np.int64 if kt == KEY_I64 else np.uint64)).view(np.uint64)
        nprop = prop.shape[0]
    rc = lib.oracle_hss(_ptr(k), _ptr(pay), N, kt, p, float(eps), int(seed) & ((1 << 64) - 1),
                        float(oversample), max_rounds, _ptr(prop), nprop, SCHEDULES[schedule], int(schedule_k),
                        _ptr(spl_key), _ptr(spl_seg), _ptr(spl_spos), _ptr(offsets),
                        _ptr(out_keys), _ptr(out_pay), ctypes.byref(st), _ptr(tl), _ptr(tu), _ptr(tr), _ptr(ts), cap)
    if rc == -1:
        raise ValueError("oracle_hss: invalid arguments")
    R = st.rounds
    res = HSSResult(
        splitter_key=(spl_key[:S].view(np.int64) if kt == KEY_I64 else spl_key[:S]),
        splitter_seg=spl_seg[:S], splitter_spos=spl_spos[:S], offsets=offsets,
        rounds=R, status=st.status, tol=st.tol,
        sample_size=np.array(st.sample_size[:R], dtype=np.uint64),
        gamma=np.array(st.gamma[:R], dtype=np.uint64),
        unresolved=np.array(st.unresolved[:R + 1], dtype=np.uint64),
    )
    if sort:
        ok = out_keys[:N]
        res.out_keys = ok.view(np.int64) if kt == KEY_I64 else ok
        res.out_payload = None if out_pay is None else out_pay[:N]
    if trace:
        res.trace_lrank = tl[:(R + 1) * S].reshape(R + 1, S)
        res.trace_urank = tu[:(R + 1) * S].reshape(R + 1, S)
        res.trace_resolved = tr[:(R + 1) * S].reshape(R + 1, S)
        used = 0
        for r in range(R):
            z = int(res.sample_size[r])
            take = min(z, max(cap - used, 0))
            blk = ts[3 * used:3 * (used + take)].reshape(take, 3)
            res.samples.append(blk.copy())
            used += take
    return res


def hss_groups(keys, p: int, nb: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 64,
               payload=None, exchange_only: bool = True):
    """The partition step of one stage of multi-stage HSS (Sec. 5.3): the p
    processors' keys split into nb buckets (nb - 1 splitters at ranks i N / nb,
    tolerance floor(N eps / (2 nb)), s nb probes per round), then the data
    exchange: bucket b is the concatenation of its runs in processor order
    (exchange_only; else each bucket is also merged)."""
    lib = _load()
    k, kt = _keys_u64(keys)
    N = int(k.shape[0])
    S = max(nb - 1, 0)
    spl_key = np.zeros(max(S, 1), dtype=np.uint64)
    spl_seg = np.zeros(max(S, 1), dtype=np.int32)
    spl_spos = np.zeros(max(S, 1), dtype=np.uint32)
    offsets = np.zeros(nb + 1, dtype=np.uint64)
    pay = None if payload is None else np.ascontiguousarray(payload, dtype=np.uint32)
    out_keys = np.empty(max(N, 1), dtype=np.uint64)
    out_pay = np.empty(max(N, 1), dtype=np.uint32) if payload is not None else None
    st = _Stats()
    rc = lib.oracle_hss_groups(_ptr(k), _ptr(pay), N, kt, p, nb, int(exchange_only), float(eps),
                               int(seed) & ((1 << 64) - 1), float(oversample), max_rounds, None, 0, 0, 0,
                               _ptr(spl_key), _ptr(spl_seg), _ptr(spl_spos), _ptr(offsets), _ptr(out_keys),
                               _ptr(out_pay), ctypes.byref(st), None, None, None, None, 0)
    if rc == -1:
        raise ValueError("oracle_hss_groups: invalid arguments")
    R = st.rounds
    res = HSSResult(
        splitter_key=(spl_key[:S].view(np.int64) if kt == KEY_I64 else spl_key[:S]),
        splitter_seg=spl_seg[:S], splitter_spos=spl_spos[:S], offsets=offsets, rounds=R, status=st.status,
        tol=st.tol, sample_size=np.array(st.sample_size[:R], dtype=np.uint64),
        gamma=np.array(st.gamma[:R], dtype=np.uint64), unresolved=np.array(st.unresolved[:R + 1], dtype=np.uint64))
    ok = out_keys[:N]
    res.out_keys = ok.view(np.int64) if kt == KEY_I64 else ok
    res.out_payload = None if out_pay is None else out_pay[:N]
    return res


@dataclass
class TwoStageResult:
    offsets: np.ndarray          # p + 1 bucket offsets of the final buckets
    out_keys: np.ndarray
    out_payload: np.ndarray | None
    stage1: HSSResult            # the r-group partition
    stage2: list                 # HSSResult of every group


def hss_two_stage(keys, p: int, r: int, eps: float, seed: int, oversample: float = 5.0, max_rounds: int = 64,
                  payload=None) -> TwoStageResult:
    """Two-stage HSS (Sec. 5.3; Sec. 7.3 runs 2 stages with r = sqrt(p)
    groups and eps per stage): stage 1 splits the p processors' keys into r
    groups with HSS (r - 1 splitters) and exchanges them; each group's
    exchanged keys (its runs in processor order) are then dealt evenly to its
    p / r processors by position, and stage 2 sorts group g with single-stage
    HSS on them, seed + 1 + g.  The final buckets are the groups' buckets in
    group order; the output is the stable sort of the input."""
    if r < 1 or p % r != 0:
        raise ValueError("r must divide p")
    pg = p // r
    st1 = hss_groups(keys, p, r, eps, seed, oversample, max_rounds, payload, exchange_only=True)
    k, kt = _keys_u64(keys)
    gk = st1.out_keys
    gp = st1.out_payload
    offsets = [0]
    outs, outp, st2 = [], [], []
    for g in range(r):
        a, b = int(st1.offsets[g]), int(st1.offsets[g + 1])
        res = hss(gk[a:b], pg, eps, seed + 1 + g, oversample=oversample, max_rounds=max_rounds,
                  payload=None if gp is None else gp[a:b])
        st2.append(res)
        outs.append(res.out_keys)
        if gp is not None:
            outp.append(res.out_payload)
        offsets.extend(int(a + x) for x in res.offsets[1:])
    out_keys = np.concatenate(outs) if outs else gk[:0]
    out_pay = np.concatenate(outp) if gp is not None and outp else None
    return TwoStageResult(offsets=np.array(offsets, dtype=np.uint64), out_keys=out_keys, out_payload=out_pay,
                          stage1=st1, stage2=st2)
