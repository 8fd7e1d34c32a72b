"""Parity of the proposal entry points (hss_partition_with_proposal,
hss_sort_with_proposal) with the oracle run on the same proposed cuts.

A proposed cut is a non-member cut (k, -1): it sorts before every input key
equal to k and its rank is #keys < k.  Before round 1 the oracle ranks every
proposed cut and offers it to every splitter's L/U (Sec. 4.2.2 steps 2-3),
so the rounds, sample sizes, |gamma|, splitters, offsets and the sorted
output must agree bit for bit.
"""
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


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def _cmp(res, ref):
    assert res.status == ref.status
    assert res.rounds == ref.rounds
    assert res.sample_size == [int(x) for x in ref.sample_size]
    assert res.gamma == [int(x) for x in ref.gamma]
    assert res.unresolved == [int(x) for x in ref.unresolved]
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    k, s, sp = res.splitter_tags()
    want_k = ref.splitter_key.view(np.uint64) if ref.splitter_key.dtype == np.int64 else ref.splitter_key
    assert np.array_equal(k.view(np.uint64), want_k)
    assert np.array_equal(s, ref.splitter_seg)
    assert np.array_equal(sp, ref.splitter_spos)


def _proposals(kind, keys, p, seed):
    g = np.random.default_rng(seed)
    srt = np.sort(keys)
    N = keys.shape[0]
    if kind == "exact":  # the ideal splitter keys: every splitter resolved before sampling
        return srt[[(i * N) // p for i in range(1, p)]]
    if kind == "noisy":  # near-quantile keys, as a decent model would give
        idx = np.clip(np.array([(i * N) // p for i in range(1, p)]) + g.integers(-N // (4 * p), N // (4 * p), p - 1),
                      0, N - 1)
        return srt[idx]
    if kind == "random":  # keys unrelated to the data, unsorted, with repeats
        r = g.integers(0, 2**63, size=2 * p, dtype=np.uint64) * np.uint64(2)
        return np.concatenate([r, r[:5]])
    if kind == "edges":  # below the minimum, above the maximum, equal to existing keys, repeated
        return np.array([0, 0, srt[0], srt[-1], np.uint64(2**64 - 1), srt[N // 2], srt[N // 2], srt[N // 3]],
                        dtype=np.uint64)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["exact", "noisy", "random", "edges"])
@pytest.mark.parametrize("N,p,eps,gen", [(1 << 16, 32, 0.02, "uniform"), (1 << 18, 64, 0.05, "zipf"),
                                         (200003, 9, 0.01, "gauss_mix")])
def test_partition_with_proposal_matches_oracle(hss, kind, N, p, eps, gen):
    keys = {"uniform": inputs.uniform, "zipf": inputs.zipf, "gauss_mix": inputs.gauss_mix}[gen](N, 4)
    prop = _proposals(kind, keys, p, 7)
    res, _ = hss.partition_with_proposal(dev(keys), p, eps, 3, dev(prop))
    ref = oracle.hss(keys, p, eps, 3, sort=False, proposal=prop)
    _cmp(res, ref)
    if kind == "exact" and gen == "uniform":
        assert res.rounds == 0


def test_sort_with_proposal_matches_oracle(hss):
    N, p, eps, seed = 1 << 18, 16, 0.02, 5
    keys = inputs.gauss_mix(N, seed)
    pay = np.arange(N, dtype=np.uint32)
    prop = _proposals("noisy", keys, p, 1)
    res = hss.sort_with_proposal(dev(keys), p, eps, seed, dev(prop), payload=dev(pay))
    ref = oracle.hss(keys, p, eps, seed, payload=pay, proposal=prop)
    _cmp(res, ref)
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys)
    assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


def test_proposal_signed_keys(hss):
    N, p, eps, seed = 1 << 17, 8, 0.02, 2
    keys = inputs.uniform(N, 6).view(np.int64)
    srt = np.sort(keys)
    prop = np.concatenate([srt[[(i * N) // p for i in range(1, p)]] + 1, np.array([-(2**63), 2**63 - 1, 0], np.int64)])
    res = hss.sort_with_proposal(torch.from_numpy(keys).cuda(), p, eps, seed, torch.from_numpy(prop).cuda(),
                                 key_type="i64")
    ref = oracle.hss(keys, p, eps, seed, proposal=prop)
    _cmp(res, ref)
    assert np.array_equal(res.keys.cpu().numpy(), ref.out_keys)


def test_empty_proposal_is_plain_partition(hss):
    N, p, eps, seed = 1 << 16, 16, 0.05, 8
    keys = inputs.uniform(N, 8)
    res, _ = hss.partition_with_proposal(dev(keys), p, eps, seed, None)
    base, _ = hss.partition(dev(keys), p, eps, seed)
    assert res.rounds == base.rounds and res.sample_size == base.sample_size
    assert torch.equal(res.offsets, base.offsets) and torch.equal(res.splitters, base.splitters)


def test_proposal_over_capacity_is_rejected(hss):
    N, p = 5000, 4
    keys = inputs.uniform(N, 1)
    prop = inputs.uniform(N + 1, 2)  # more cuts than the round sample capacity min(N, ...)
    with pytest.raises(RuntimeError):
        hss.partition_with_proposal(dev(keys), p, 0.05, 1, dev(prop))


def test_proposal_when_every_splitter_starts_resolved(hss):
    """eps so large that the sentinels already satisfy every splitter: no
    round runs, but the proposed cuts still improve L/U and so the final
    splitters (the closer of L and U)."""
    N, p, eps, seed = 1 << 14, 4, 4.0, 1
    keys = inputs.uniform(N, 2)
    prop = np.sort(keys)[[N // 4 + 3, N // 2 - 7, (3 * N) // 4]]
    res, _ = hss.partition_with_proposal(dev(keys), p, eps, seed, dev(prop))
    ref = oracle.hss(keys, p, eps, seed, sort=False, proposal=prop)
    _cmp(res, ref)
    assert res.rounds == 0
