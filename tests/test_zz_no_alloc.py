"""hss_local_sort_noalloc: the local sort for callers that cannot allocate.

Some callers of this library may not allocate device memory at all, for
instance code that runs inside a host framework owning every allocation or a
thread that must not take the allocator's locks.  hss_local_sort_noalloc
serves them from a fixed scratch array inside the library.  These tests call
it through the C ABI and check that it returns exactly what the regular
hss_local_sort returns (integer sort: bit for bit), on two calls in a row,
that it equals the CPU oracle's stable local sort, and that inputs past its
fixed limit are refused before any device work.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HSS_ERR_NOALLOC_LIMIT = -7
MAX_KEYS = 1 << 19


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_1803_01237_gb300 import hss
    L = hss.load()
    f = L.hss_local_sort_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P, P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, P, P, P]
    f.restype = ctypes.c_int
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(lib, keys, p, payload=None, key_type=0):
    out = torch.empty_like(keys)
    outp = torch.empty_like(payload) if payload is not None else None
    rc = lib.hss_local_sort_noalloc(_ptr(keys), _ptr(payload), key_type, keys.numel(), p, _ptr(out), _ptr(outp),
                                    _stream())
    return rc, out, outp


@pytest.mark.parametrize("N,p,payload,key_type", [(MAX_KEYS, 8, True, 0), (100003, 3, False, 1),
                                                  (60000, 4, True, 0), (5000, 64, False, 0)])
def test_noalloc_matches_local_sort_twice(lib, N, p, payload, key_type):
    from paper_1803_01237_gb300 import hss
    kt = "i64" if key_type else "u64"
    for call in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
        keys = torch.from_numpy(inputs.zipf(N, 10 * N + call, distinct=1000).view(np.int64)).cuda()
        pay = torch.from_numpy((np.arange(N, dtype=np.uint32) * np.uint32(7 + call)).view(np.int32)).cuda() \
            if payload else None
        rc, out, outp = _noalloc(lib, keys, p, pay, key_type)
        assert rc == 0, rc
        if payload:
            ref, refp = hss.local_sort(keys, p, payload=pay, key_type=kt)
            assert torch.equal(outp, refp)
        else:
            ref = hss.local_sort(keys, p, key_type=kt)
        assert torch.equal(out, ref)


def test_noalloc_refuses_oversized_inputs(lib):
    keys = torch.zeros(MAX_KEYS + 1, dtype=torch.int64, device="cuda")
    rc, _, _ = _noalloc(lib, keys, 4)
    assert rc == HSS_ERR_NOALLOC_LIMIT
    keys = torch.zeros(1000, dtype=torch.int64, device="cuda")
    rc, _, _ = _noalloc(lib, keys, 1 << 20)  # segment bookkeeping past the fixed scratch
    assert rc == HSS_ERR_NOALLOC_LIMIT


def test_noalloc_allocates_nothing(lib):
    """The call leaves torch's allocator untouched (no device allocation)."""
    N, p = 200000, 4
    keys = torch.from_numpy(inputs.uniform(N, 3).view(np.int64)).cuda()
    out = torch.empty_like(keys)
    # first use on this device loads the library's device image (with its
    # fixed scratch array); measure after that
    assert lib.hss_local_sort_noalloc(_ptr(keys), None, 0, N, p, _ptr(out), None, _stream()) == 0
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free_before, _ = torch.cuda.mem_get_info()
    rc = lib.hss_local_sort_noalloc(_ptr(keys), None, 0, N, p, _ptr(out), None, _stream())
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert rc == 0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
    assert free_after >= free_before - (2 << 20)  # no new device memory beyond driver noise


@pytest.mark.parametrize("N,p,key_type", [(70001, 5, 0), (4096, 16, 1)])
def test_noalloc_matches_oracle(lib, N, p, key_type):
    """Against the oracle's stable local sort of every segment (Sec. 6.1
    tagging): keys and the payload (each key's input index) bit for bit."""
    raw = inputs.zipf(N, 77 + N, distinct=500)
    keys_h = raw.view(np.int64) if key_type else raw
    pay_h = np.arange(N, dtype=np.uint32)
    ref_k, ref_p = oracle.segment_sort(keys_h, p, payload=pay_h)
    keys = torch.from_numpy(raw.view(np.int64)).cuda()
    pay = torch.from_numpy(pay_h.view(np.int32)).cuda()
    rc, out, outp = _noalloc(lib, keys, p, pay, key_type)
    assert rc == 0, rc
    assert np.array_equal(out.cpu().numpy().view(np.uint64), np.ascontiguousarray(ref_k).view(np.uint64))
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), ref_p)


def test_noalloc_refuses_a_capturing_stream(lib):
    """The call reads its status word back with a stream synchronisation; on a
    stream that is capturing work it returns HSS_ERR_INVALID without enqueuing."""
    N, p = 1000, 2
    keys = torch.from_numpy(inputs.uniform(N, 5).view(np.int64)).cuda()
    out = torch.empty_like(keys)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            rc = lib.hss_local_sort_noalloc(_ptr(keys), None, 0, N, p, _ptr(out), None,
                                            ctypes.c_void_p(s.cuda_stream))
        finally:
            g.capture_end()
    assert rc == -1
    # the stream and the library stay usable
    rc, out2, _ = _noalloc(lib, keys, p)
    assert rc == 0
