"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without a
GPU, exports every function include/hss.h declares, sizes workspaces and
rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hss.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1803_01237_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hss_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_functions()
    for must in ("hss_partition", "hss_sort", "hss_local_sort", "hss_rank_cuts", "hss_exchange", "hss_merge",
                 "hss_workspace_bytes", "hss_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_built_for_sm_103a():
    from paper_1803_01237_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_strerror(lib):
    lib.hss_strerror.restype = ctypes.c_char_p
    lib.hss_strerror.argtypes = [ctypes.c_int]
    assert lib.hss_strerror(0) == b"ok"
    assert b"workspace" in lib.hss_strerror(-2)
    assert lib.hss_strerror(12345) == b"unknown error"


def test_workspace_sizes_grow_with_n():
    from paper_1803_01237_gb300 import hss
    a = hss.workspace_bytes("sort", 1 << 20, 64)
    b = hss.workspace_bytes("sort", 1 << 22, 64)
    assert 0 < a < b
    assert hss.workspace_bytes("sort", 1 << 20, 64, payload=True) > a
    assert hss.workspace_bytes("partition", 1 << 20, 64) <= a
    # the sort keeps two key buffers of N u64 at least
    assert a >= 2 * 8 * (1 << 20)


def test_invalid_arguments_rejected_without_device(lib):
    from paper_1803_01237_gb300 import hss
    L = hss.load()
    st = hss.Stats()
    bad = [hss.Params(eps=0.0, seed=1, p=4, oversample=5.0, max_rounds=0, flags=0),
           hss.Params(eps=0.05, seed=1, p=0, oversample=5.0, max_rounds=0, flags=0),
           hss.Params(eps=float("nan"), seed=1, p=4, oversample=5.0, max_rounds=0, flags=0),
           hss.Params(eps=0.05, seed=1, p=4, oversample=0.0, max_rounds=0, flags=0),
           hss.Params(eps=0.05, seed=1, p=4, oversample=5.0, max_rounds=65, flags=0),
           hss.Params(eps=0.05, seed=1, p=4, oversample=5.0, max_rounds=0, flags=0, schedule=3),
           hss.Params(eps=0.05, seed=1, p=4, oversample=5.0, max_rounds=0, flags=0, schedule=1, schedule_k=0),
           hss.Params(eps=0.05, seed=1, p=4, oversample=5.0, max_rounds=0,
                      flags=hss.FLAG_HIST_PROBE | hss.FLAG_HIST_STAGED)]
    dummy = ctypes.c_void_p(16)
    for prm in bad:
        rc = L.hss_partition(dummy, 0, 100, ctypes.byref(prm), dummy, dummy, dummy, 1 << 30, ctypes.byref(st), None)
        assert rc == -1
    ok = hss.Params(eps=0.05, seed=1, p=4, oversample=5.0, max_rounds=0, flags=0)
    # workspace too small
    rc = L.hss_partition(dummy, 0, 100, ctypes.byref(ok), dummy, dummy, dummy, 16, ctypes.byref(st), None)
    assert rc == -2
    # bad key type
    rc = L.hss_partition(dummy, 7, 100, ctypes.byref(ok), dummy, dummy, dummy, 1 << 30, ctypes.byref(st), None)
    assert rc == -1
    # null keys with N > 0
    rc = L.hss_partition(None, 0, 100, ctypes.byref(ok), dummy, dummy, dummy, 1 << 30, ctypes.byref(st), None)
    assert rc == -1
    # payload without an output payload
    rc = L.hss_sort(dummy, dummy, 0, 100, ctypes.byref(ok), dummy, None, dummy, dummy, dummy, 1 << 30,
                    ctypes.byref(st), None)
    assert rc == -1
    # local sort: p = 0
    rc = L.hss_local_sort(dummy, None, 0, 100, 0, dummy, None, dummy, 1 << 30, None)
    assert rc == -1
    # sample words: range past 2^32
    rc = L.hss_sample_words(1, 0, 1, 0xFFFFFFFF, 2, dummy, None)
    assert rc == -1


def test_no_cpu_fallback_in_binding():
    """The binding is marshalling only: it never imports the oracle."""
    src = open(os.path.join(ROOT, "paper_1803_01237_gb300", "hss.py")).read()
    assert "oracle" not in src.replace("# ", "")
    for f in os.listdir(os.path.join(ROOT, "paper_1803_01237_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_1803_01237_gb300", "csrc", f)).read().lower()


def test_binding_rejects_host_tensors_before_any_device_call():
    """Device entry points refuse host data up front (no host pointer ever
    reaches a kernel); the host entry point is sort_host."""
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss
    cpu = torch.zeros(16, dtype=torch.int64)
    with pytest.raises(ValueError):
        hss.sort(cpu, 2, 0.05, 1)
    with pytest.raises(ValueError):
        hss.partition(cpu, 2, 0.05, 1)
    with pytest.raises(ValueError):
        hss.local_sort(cpu, 2)
    with pytest.raises(TypeError):
        hss.sort(np.zeros(16, dtype=np.uint64), 2, 0.05, 1)
    with pytest.raises(ValueError):
        hss._ptr(cpu)
    assert hss._ptr(np.zeros(4, dtype=np.uint64)) is not None


def test_segment_size_limit_rejected_without_device(lib):
    """A segment or bucket of 2^30 keys or more would overflow the split's
    30-bit look-back counts: every entry point refuses it up front."""
    from paper_1803_01237_gb300 import hss
    L = hss.load()
    st = hss.Stats()
    dummy = ctypes.c_void_p(16)
    big = 1 << 31
    prm = hss.Params(eps=0.05, seed=1, p=1, oversample=5.0, max_rounds=0, flags=0)
    assert L.hss_local_sort(dummy, None, 0, big, 1, dummy, None, dummy, 1 << 62, None) == -1
    assert L.hss_partition(dummy, 0, big, ctypes.byref(prm), dummy, dummy, dummy, 1 << 62, ctypes.byref(st), None) == -1
    assert L.hss_sort(dummy, None, 0, big, ctypes.byref(prm), dummy, None, dummy, dummy, dummy, 1 << 62,
                      ctypes.byref(st), None) == -1
    assert L.hss_rank_cuts(dummy, 0, big, 1, dummy, 1, dummy, None, None) == -1
    assert L.hss_exchange(dummy, None, big, 1, dummy, dummy, dummy, None, dummy, 1 << 62, None) == -1
    # a segment just below the limit passes the size check (and fails on the workspace)
    n_ok = (1 << 30) - 1
    assert L.hss_local_sort(dummy, None, 0, n_ok, 1, dummy, None, dummy, 16, None) == -2
    # the sorting calls also bound the eps-balanced buckets: 2^30 - 1 keys on one
    # processor is fine, but two processors of 2^29 + eps slack are not at large eps
    prm2 = hss.Params(eps=1.0, seed=1, p=2, oversample=5.0, max_rounds=0, flags=0)
    assert L.hss_sort(dummy, None, 0, 1 << 30, ctypes.byref(prm2), dummy, None, dummy, dummy, dummy, 1 << 62,
                      ctypes.byref(st), None) == -1


def test_two_stage_arguments_rejected_without_device(lib):
    """hss_sort_two_stage sizes its workspace on the host and refuses group
    counts that do not divide p, a single group, fewer than 2p keys and
    schedules other than the proportional one before any device work."""
    from paper_1803_01237_gb300 import hss
    L = hss.load()
    L.hss_two_stage_workspace_bytes.restype = ctypes.c_size_t
    L.hss_two_stage_workspace_bytes.argtypes = [ctypes.c_uint64, ctypes.POINTER(hss.Params), ctypes.c_uint32,
                                                ctypes.c_int, ctypes.c_int]

    def prm(p, **kw):
        return hss.Params(eps=kw.get("eps", 0.02), seed=1, p=p, oversample=5.0, max_rounds=0, flags=0,
                          schedule=kw.get("schedule", 0))

    N = 1 << 20
    ok = L.hss_two_stage_workspace_bytes(N, ctypes.byref(prm(256)), 16, 0, 0)
    assert ok >= 2 * 8 * N
    assert L.hss_two_stage_workspace_bytes(N, ctypes.byref(prm(256)), 16, 0, 1) > ok
    assert L.hss_two_stage_workspace_bytes(N << 1, ctypes.byref(prm(256)), 16, 0, 0) > ok
    for n, p, r, kw in [(N, 256, 1, {}), (N, 256, 24, {}), (N, 256, 512, {}), (300, 256, 16, {}),
                        (N, 256, 16, {"schedule": 1}), (N, 256, 16, {"eps": 0.0}), (N, 1 << 18, 2, {})]:
        assert L.hss_two_stage_workspace_bytes(n, ctypes.byref(prm(p, **kw)), r, 0, 0) == 0
    # a group at its balance bound reaches 2^30 keys with 2^31 keys in 2 groups, not in 8
    assert L.hss_two_stage_workspace_bytes(1 << 31, ctypes.byref(prm(8)), 2, 0, 0) == 0
    assert L.hss_two_stage_workspace_bytes(1 << 31, ctypes.byref(prm(8)), 8, 0, 0) > 0
    P = ctypes.c_void_p
    L.hss_sort_two_stage.restype = ctypes.c_int
    L.hss_sort_two_stage.argtypes = [P, P, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(hss.Params), ctypes.c_uint32,
                                     P, P, P, P, P, P, ctypes.c_size_t, ctypes.POINTER(hss.TwoStageStats), P, P]
    st = hss.TwoStageStats()
    dummy = ctypes.c_void_p(16)
    args = lambda p, r, work: (dummy, None, 0, N, ctypes.byref(prm(p)), r, dummy, None, dummy, dummy, dummy, dummy,
                               work, ctypes.byref(st), None, None)
    assert L.hss_sort_two_stage(*args(256, 24, 1 << 40)) == -1
    assert L.hss_sort_two_stage(*args(256, 16, 16)) == -2


def test_cut_records_match_the_c_layout():
    """The binding's packed (n, 2) int64 cut tensors hold hss_cut records
    byte for byte (u64 key, i32 seg, u32 spos: 16 bytes, little-endian), the
    special segs -1/-2/-3 and positions above 2^31 included, both ways."""
    import torch
    from paper_1803_01237_gb300 import hss

    class Cut(ctypes.Structure):
        _fields_ = [("key", ctypes.c_uint64), ("seg", ctypes.c_int32), ("spos", ctypes.c_uint32)]

    assert ctypes.sizeof(Cut) == 16
    vals = [(0, 0, 0), ((1 << 64) - 1, 7, (1 << 32) - 1), (5, -1, 0), (0, -2, 0), (0, -3, 0),
            (1 << 63, (1 << 31) - 1, 1 << 31), (12345, 3, 99)]
    arr = (Cut * len(vals))(*[Cut(*v) for v in vals])
    raw = bytes(arr)
    key = np.array([v[0] for v in vals], dtype=np.uint64)
    seg = np.array([v[1] for v in vals], dtype=np.int32)
    spos = np.array([v[2] for v in vals], dtype=np.uint32)
    packed = hss.cuts_from_numpy(key, seg, spos, "cpu")
    assert packed.shape == (len(vals), 2) and packed.dtype == torch.int64
    assert packed.numpy().tobytes() == raw
    k, s, sp = hss.cuts_to_numpy(torch.from_numpy(np.frombuffer(raw, dtype=np.int64).copy()).reshape(-1, 2))
    assert np.array_equal(k.view(np.uint64), key) and np.array_equal(s, seg) and np.array_equal(sp, spos)


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors with ctypes has the size and field
    offsets that a C compiler gives the header's declaration (gcc, host ABI)."""
    import subprocess
    from paper_1803_01237_gb300 import hss
    mirrors = {"hss_params": hss.Params, "hss_stats": hss.Stats, "hss_tuning": hss.Tuning,
               "hss_job_stats": hss.JobStats, "hss_batch_stats": hss.BatchStats,
               "hss_two_stage_stats": hss.TwoStageStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hss.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    # CDFModel reads theta at byte 0 and the Adam step counter at byte 12 NPARAM of hss_cdf_model
    lines.append('    printf("hss_cdf_model size %zu\\n", sizeof(hss_cdf_model));')
    for fld in ("theta", "step"):
        lines.append(f'    printf("hss_cdf_model {fld} %zu\\n", offsetof(hss_cdf_model, {fld}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, v = line.split()
        got[(cname, field)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
    lib = hss.load()
    lib.hss_cdf_model_bytes.restype = ctypes.c_size_t
    assert got[("hss_cdf_model", "size")] == lib.hss_cdf_model_bytes()
    assert got[("hss_cdf_model", "theta")] == 0 and got[("hss_cdf_model", "step")] == 12 * hss.CDF_NPARAM


def test_binding_constants_match_the_header():
    """Error codes, key types, operations, flags, limits, schedules and the
    CDF network's constants in the binding equal the header's #defines."""
    from paper_1803_01237_gb300 import hss
    defs = {}
    for m in re.finditer(r"^#define\s+(HSS_\w+)\s+\(?(-?\d+)u?\)?", open(HEADER).read(), re.M):
        defs[m.group(1)] = int(m.group(2))
    want = {"HSS_ERR_INVALID": hss.ERR_INVALID, "HSS_ERR_WORKSPACE": hss.ERR_WORKSPACE,
            "HSS_ERR_ROUND_LIMIT": hss.ERR_ROUND_LIMIT, "HSS_ERR_TIMEOUT": hss.ERR_TIMEOUT,
            "HSS_ERR_CUDA": hss.ERR_CUDA, "HSS_ERR_CAPACITY": hss.ERR_CAPACITY,
            "HSS_FLAG_SYNC": hss.FLAG_SYNC, "HSS_FLAG_TIMING": hss.FLAG_TIMING,
            "HSS_FLAG_HIST_PROBE": hss.FLAG_HIST_PROBE, "HSS_FLAG_HIST_STAGED": hss.FLAG_HIST_STAGED,
            "HSS_FLAG_HOST_ROUNDS": hss.FLAG_HOST_ROUNDS, "HSS_FLAG_DEVICE_ROUNDS": hss.FLAG_DEVICE_ROUNDS,
            "HSS_MAX_ROUNDS": hss.MAX_ROUNDS, "HSS_NUM_PHASES": hss.NUM_PHASES, "HSS_CDF_NPARAM": hss.CDF_NPARAM,
            "HSS_KEY_U64": hss.KEY_TYPES["u64"], "HSS_KEY_I64": hss.KEY_TYPES["i64"],
            "HSS_CDF_LINEAR": hss.CDF_FEATURES["linear"], "HSS_CDF_LOG": hss.CDF_FEATURES["log"],
            "HSS_CDF_W_FP32": hss.CDF_WEIGHTS["fp32"], "HSS_CDF_W_BF16": hss.CDF_WEIGHTS["bf16"]}
    for name, op in [("SORT", "sort"), ("PARTITION", "partition"), ("LOCAL_SORT", "local_sort"),
                     ("MERGE", "merge"), ("EXCHANGE", "exchange"), ("SORT_HOST", "sort_host")]:
        want["HSS_OP_" + name] = hss.OP[op]
    for name in ("PROPORTIONAL", "THEORY", "EQUAL"):
        want["HSS_SCHEDULE_" + name] = hss.SCHEDULES[name.lower()]
    want["HSS_OK"] = hss.HSS_OK
    for name, v in want.items():
        assert defs[name] == v, name
    codes = {v: k for k, v in defs.items() if k.startswith("HSS_ERR_")}
    for code, name in codes.items():
        assert hss.ERRORS[code] == name
    assert set(hss.ERRORS) == set(codes)


def _header_arity():
    """Number of parameters of every hss_* prototype in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(hss_\w+)\s*\(([^;{}]*?)\)\s*;", text, re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argtypes_match_header_arity():
    """Every entry point whose argument types the binding declares (at load
    time or on first use) takes as many arguments as the header's prototype."""
    from paper_1803_01237_gb300 import hss
    lib = hss.load()
    for bind in (hss._bind_call_stats, hss._bind_batch, hss._bind_two_stage):  # bound on first use
        bind(lib)
    arity = _header_arity()
    assert len(arity) >= 30
    checked = 0
    for name, n in arity.items():
        fn = getattr(lib, name, None)
        if fn is not None and fn.argtypes is not None:
            assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
            checked += 1
    assert checked >= 28
