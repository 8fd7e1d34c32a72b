"""The CUDA path at the full sizes of the workloads, in the launch
configuration bench.py times.

The CPU oracle cannot run 2^28 keys in test time, so these tests check what
holds at any size and what the oracle can compute one item at a time:
  * the output is the stable sort of the input (against torch's stable sort
    on the device, with the payload carrying each key's input index);
  * chi(0) = 0, chi(p) = N, monotone, every |chi(i) - t_i| <= floor(N eps/2p)
    (Sec. 2), hence every bucket within the balance bound;
  * a sample of splitters: the oracle sorts only the splitter's segment and
    finds the input element at the splitter's tag; the globally sorted output
    holds that element at position chi(i) (S(i) = I(chi(i)));
  * per-round sample sizes inside a 6-sigma band of q |gamma| (Lemma 4.6).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hss():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_1803_01237_gb300 import hss as h
    h.load()
    return h


def _check_fullsize(hss, keys_h, p, eps, seed, payload_is_index=True, oversample=5.0):
    N = keys_h.shape[0]
    dk = torch.from_numpy(keys_h.view(np.int64)).cuda()
    dp = torch.arange(N, dtype=torch.int32, device="cuda") if payload_is_index else None
    res = hss.sort(dk, p, eps, seed, payload=dp, oversample=oversample)
    torch.cuda.synchronize()
    assert res.status == 0
    # 1. stable sort of the input (u64 order = i64 order after flipping the sign bit)
    sign = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    flipped = torch.bitwise_xor(dk, sign)
    ref_vals, ref_idx = torch.sort(flipped, stable=True)
    assert torch.equal(torch.bitwise_xor(res.keys, sign), ref_vals)
    if payload_is_index:
        assert torch.equal(res.payload.to(torch.int64), ref_idx)
    del flipped, ref_vals, ref_idx
    # 2. offsets within the target ranges
    off = res.offsets.cpu().numpy().astype(np.int64)
    tol = oracle.tolerance(N, p, eps)
    assert res.tol == tol
    t = (np.arange(1, p, dtype=object) * N // p).astype(np.int64)
    assert off[0] == 0 and off[-1] == N and np.all(np.diff(off) >= 0)
    assert np.all(np.abs(off[1:-1] - t) <= tol)
    # 3. sampled splitters are the input elements of rank chi(i)
    k_spl, seg, spos = res.splitter_tags()
    out_pay = res.payload.cpu().numpy() if payload_is_index else None
    out_keys = res.keys.cpu().numpy().view(np.uint64)
    bounds = oracle.segment_bounds(N, p)
    g = np.random.default_rng(seed)
    for i in g.choice(p - 1, size=min(12, p - 1), replace=False):
        s = int(seg[i])
        assert s >= 0
        lo, hi = int(bounds[s]), int(bounds[s + 1])
        srt, idx = oracle.segment_sort(keys_h[lo:hi], 1, payload=np.arange(lo, hi, dtype=np.uint32))
        assert srt[int(spos[i])] == np.uint64(k_spl[i])
        assert out_keys[int(off[i + 1])] == np.uint64(k_spl[i])
        if payload_is_index:
            assert int(out_pay[int(off[i + 1])]) == int(idx[int(spos[i])])
    # 4. sample sizes inside a Chernoff band around q |gamma|
    for r in range(res.rounds):
        gam = res.gamma[r]
        q = min(1.0, oversample * p / gam)
        mean = q * gam
        sd = math.sqrt(max(mean * (1 - q), 1e-9))
        assert abs(res.sample_size[r] - mean) <= 6 * sd + 1
    return res


@pytest.mark.timeout(600)
@pytest.mark.parametrize("dist", ["uniform", "gauss_mix", "zipf"])
def test_bench_workload_fullsize(hss, dist):
    """N = 2^28 uint64, p = 1024, eps = 0.02: the bench configuration."""
    N = 1 << 28
    seed = {"uniform": 1, "gauss_mix": 2, "zipf": 3}[dist]
    keys = inputs.SCALE_DISTRIBUTIONS[dist](N, seed)
    res = _check_fullsize(hss, keys, 1024, 0.02, seed)
    assert res.rounds <= 12


@pytest.mark.timeout(900)
def test_plummer_morton_payload_fullsize(hss):
    """2^30 Morton keys of a Plummer sphere with the particle index as
    payload, p = 16384, eps = 0.01 (the N-body workload)."""
    N = 1 << 30
    keys, payload = inputs.plummer_morton(N, 7)
    assert np.array_equal(payload[:1000], np.arange(1000, dtype=np.uint32))
    del payload
    _check_fullsize(hss, keys, 16384, 0.01, 7)


def test_exact_splitting(hss):
    """eps = p/N makes the half-width floor(1/2) = 0: exact splitting (the
    eps = p/N case after Theorem 4.8): every bucket holds N/p keys."""
    N, p = 1 << 22, 256
    keys = inputs.uniform(N, 21)
    res = _check_fullsize(hss, keys, p, p / N, 21)
    assert res.tol == 0
    off = res.offsets.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(off) == N // p)
    ref = oracle.hss(keys[: 1 << 16], 64, 64 / (1 << 16), 21, sort=False)
    small = hss.sort(torch.from_numpy(keys[: 1 << 16].view(np.int64)).cuda(), 64, 64 / (1 << 16), 21)
    assert small.rounds == ref.rounds and small.sample_size == [int(x) for x in ref.sample_size]
    assert np.array_equal(small.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
