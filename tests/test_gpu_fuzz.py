"""Seeded random cases against the oracle: sizes, processor counts, eps,
oversampling, key types, payloads, distributions and the entry points
(single-stage sort and partition, two-stage sort, batches) drawn at random,
each compared bit for bit.  The draws are fixed by the test's seed, so a
failure names a reproducible case."""
import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GENS = [inputs.uniform, inputs.gauss_mix, inputs.zipf, inputs.skew1, inputs.skew2, inputs.skew3, inputs.gauss,
        inputs.nested_clusters, lambda n, s: inputs.lognormal_job(n, s), lambda n, s: inputs.allzeros(n)]


@pytest.fixture(scope="module")
def hss():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_1803_01237_gb300 import hss as h
    h.load()
    return h


def _draw(case):
    g = np.random.default_rng(1000 + case)
    N = int(g.integers(1, 1 << 17))
    p = int(min(N, 2 ** g.integers(0, 10) + g.integers(0, 3)))
    eps = float(g.choice([0.005, 0.01, 0.03, 0.1, 0.5]))
    s = float(g.choice([1.0, 2.0, 5.0, 9.0]))
    seed = int(g.integers(0, 1 << 63))
    kt = "i64" if g.random() < 0.3 else "u64"
    pay = g.random() < 0.5
    gen = GENS[int(g.integers(0, len(GENS)))]
    keys = gen(N, int(g.integers(1, 1000)))
    if kt == "i64":
        keys = (keys.view(np.int64) - np.int64(int(g.integers(0, 1 << 62)))).astype(np.int64)
    payload = (np.arange(N, dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32) if pay else None
    return N, max(p, 1), eps, s, seed, kt, keys, payload


@pytest.mark.parametrize("case", range(40))
def test_random_sort_matches_oracle(hss, case):
    N, p, eps, s, seed, kt, keys, payload = _draw(case)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(payload.view(np.int32)).cuda() if payload is not None else None
    res = hss.sort(dk, p, eps, seed, payload=dp, oversample=s, key_type=kt)
    ref = oracle.hss(keys, p, eps, seed, oversample=s, payload=payload)
    assert res.rounds == ref.rounds and res.status == ref.status
    assert res.sample_size == [int(x) for x in ref.sample_size]
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    if p > 1:
        k, sg, sp = hss.cuts_to_numpy(res.splitters)
        want = ref.splitter_key.view(np.uint64) if ref.splitter_key.dtype == np.int64 else ref.splitter_key
        assert np.array_equal(k.view(np.uint64), want)
        assert np.array_equal(sg, ref.splitter_seg) and np.array_equal(sp, ref.splitter_spos)
    out = res.keys.cpu().numpy()
    assert np.array_equal(out.view(np.uint64), ref.out_keys.view(np.uint64))
    if payload is not None:
        assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


@pytest.mark.parametrize("case", range(12))
def test_random_two_stage_matches_oracle(hss, case):
    N, p, eps, s, seed, kt, keys, payload = _draw(500 + case)
    g = np.random.default_rng(77 + case)
    r = int(2 ** g.integers(1, 5))
    p = r * int(2 ** g.integers(0, 5))
    N = max(N, 2 * p)
    keys = inputs.gauss_mix(N, case + 3)
    payload = None if payload is None else (np.arange(N, dtype=np.uint64) % (1 << 32)).astype(np.uint32)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(payload.view(np.int32)).cuda() if payload is not None else None
    ref = oracle.hss_two_stage(keys, p, r, eps, seed, oversample=s, payload=payload)
    if any(int(ref.stage1.offsets[j + 1] - ref.stage1.offsets[j]) < p // r for j in range(r)):
        pytest.skip("a group smaller than its processor count (refused by the device entry point)")
    res = hss.sort_two_stage(dk, p, r, eps, seed, payload=dp, oversample=s)
    assert res.stage1.rounds == ref.stage1.rounds
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys.view(np.uint64))
    if payload is not None:
        assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


@pytest.mark.parametrize("case", range(6))
def test_random_batch_matches_oracle(hss, case):
    g = np.random.default_rng(900 + case)
    nj = int(g.integers(1, 24))
    sizes = [int(g.integers(0, 40000)) for _ in range(nj)]
    ps = [int(max(1, min(max(n, 1), g.integers(1, 200)))) for n in sizes]
    seeds = [int(g.integers(0, 1 << 62)) for _ in range(nj)]
    eps = float(g.choice([0.01, 0.05, 0.2]))
    jobs = [GENS[int(g.integers(0, len(GENS)))](n, j + 5) for j, n in enumerate(sizes)]
    keys = np.concatenate(jobs) if nj else np.zeros(0, dtype=np.uint64)
    res = hss.sort_batch(torch.from_numpy(keys.view(np.int64)).cuda(), sizes, ps, eps, 0, seeds=seeds)
    out = res.keys.cpu().numpy().view(np.uint64)
    o = 0
    for j, (n, p) in enumerate(zip(sizes, ps)):
        ref = oracle.hss(jobs[j], p, eps, seeds[j])
        assert res.job_rounds[j] == ref.rounds
        assert np.array_equal(res.job_offsets(j).cpu().numpy().astype(np.uint64), ref.offsets)
        assert np.array_equal(out[o:o + n], ref.out_keys.view(np.uint64))
        o += n
