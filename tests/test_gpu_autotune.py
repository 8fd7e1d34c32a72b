"""The autotuner on the GPU: it measures a space of choices and caches the
fastest, and none of the tiling choices changes a result -- every one gives
the oracle's splitters, offsets and sorted keys (the oversampling s it picks
is the s the oracle is run with)."""
import functools

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
    yield h
    h.reset_tuning()


_GENS = {"uniform": inputs.uniform, "gauss_mix": inputs.gauss_mix, "zipf": inputs.zipf,
         "nested": inputs.nested_clusters}


@functools.lru_cache(maxsize=None)
def _case(gen):
    keys = _GENS[gen](1 << 21, 3)
    return keys, oracle.hss(keys, 16, 0.02, 3)


@pytest.mark.parametrize("gen", list(_GENS))
@pytest.mark.parametrize("tiling", [(4096, 0, 384), (14336, 0, 384), (4096, 1, 384), (4096, 1, 128), (14336, 1, 4096),
                                    (4096, 0, 384, 1), (4096, 0, 384, 4096), (14336, 0, 384, 4096),
                                    (4096, 0, 384, 0, 1), (14336, 1, 384, 1, 1), (4096, 0, 384, 0, 0, 1),
                                    (14336, 1, 384, 0, 0, 1), (4096, 0, 384, 0, 1, 1)])
def test_tilings_give_the_oracle_result(hss, gen, tiling):
    p, eps, seed = 16, 0.02, 3
    keys, ref = _case(gen)
    hss.set_tuning(*tiling)
    try:
        res = hss.sort(torch.from_numpy(keys.view(np.int64)).cuda(), p, eps, seed)
        torch.cuda.synchronize()
    finally:
        hss.reset_tuning()
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys)


@pytest.mark.parametrize("gen", ["uniform", "zipf", "nested"])
@pytest.mark.parametrize("split_scatter", [0, 1])
def test_split_scatter_keeps_the_payload_stable(hss, gen, split_scatter):
    """Both ways of writing a split tile give the oracle's stable sort with
    the payload in tow (equal keys keep input order)."""
    N, p, eps, seed = 1 << 20, 16, 0.02, 5
    keys = _GENS[gen](N, 9)
    pay = np.arange(N, dtype=np.uint32)
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    hss.set_tuning(split_scatter=split_scatter)
    try:
        res = hss.sort(torch.from_numpy(keys.view(np.int64)).cuda(), p, eps, seed,
                       payload=torch.from_numpy(pay.view(np.int32)).cuda())
        torch.cuda.synchronize()
    finally:
        hss.reset_tuning()
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys)
    assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


def test_tuner_picks_and_caches_a_choice(hss, tmp_path):
    from paper_1803_01237_gb300 import autotune
    t = autotune.Tuner(str(tmp_path / "t.json"))
    space = ([3.0, 8.0], [(4096, 0, 384), (4096, 1, 384)])
    N, p, eps, seed = 1 << 20, 64, 0.05, 2
    c = t.tune(N, p, eps=eps, kind="uniform", trials=1, space=space, seed=seed)
    assert c.oversample in (3.0, 8.0)
    rec = next(iter(t.cache.values()))
    assert len(rec["measured"]) == 4 + 3
    assert autotune.Tuner(str(tmp_path / "t.json")).cache == t.cache  # persisted
    assert t.tune(N, p, eps=eps, kind="uniform", space=space) == c  # from the cache
    keys = inputs.uniform(N, seed)
    s, flags = c.apply()
    try:
        res = hss.sort(torch.from_numpy(keys.view(np.int64)).cuda(), p, eps, seed, oversample=s, flags=flags)
        torch.cuda.synchronize()
    finally:
        hss.reset_tuning()
    ref = oracle.hss(keys, p, eps, seed, oversample=s)
    assert res.rounds == ref.rounds
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys)
