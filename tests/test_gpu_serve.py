"""The serving loop (continuous batching of partition requests): results do
not depend on the mix, memory admission holds, and online training of the
CDF network makes later requests start from proposals that save rounds."""
import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_1803_01237_gb300 import hss, serve
    hss.load()
    return hss, serve


def _pool(n_bufs, n, seed):
    return [torch.from_numpy(inputs.lognormal_job(n, seed + b).view(np.int64)).cuda() for b in range(n_bufs)]


def _same(a, b):
    assert a.error is None and b.error is None, (a.error, b.error)
    assert a.rounds == b.rounds
    assert torch.equal(a.offsets, b.offsets) and torch.equal(a.splitters, b.splitters)


def _check_contract(c):
    off = c.offsets.cpu().numpy().astype(np.int64)
    n, p = c.n, c.p
    t = np.array([(i * n) // p for i in range(1, p)], dtype=np.int64)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert np.all(np.abs(off[1:-1] - t) <= c.tol)


def test_results_same_alone_and_in_the_mix(mods):
    hss, serve = mods
    pool = _pool(2, 1 << 21, 40)
    reqs = serve.poisson_requests(pool, 24, rate=400.0, seed=3, lo_log2=14, hi_log2=20, ps=(64, 256))
    alone = serve.Server(slots=1).run(reqs, realtime=False)
    srv = serve.Server(slots=4)
    srv.warmup()
    mix = srv.run(reqs, realtime=True)
    assert mix.max_in_flight > 1
    for a, b in zip(alone.completions, mix.completions):
        assert a.rid == b.rid
        _same(a, b)
        _check_contract(b)


def test_frozen_model_proposals_same_alone_and_in_the_mix(mods):
    hss, serve = mods
    pool = _pool(2, 1 << 21, 50)
    # pre-train on one job's splitters
    keys = pool[0]
    m = hss.CDFModel().init(2, "log", 1, (1 << 63) - 1)
    res, _ = hss.partition(keys, 512, 0.02, 1)
    tk, tr = hss.training_pairs(res)
    m.train(tk, tr, keys.numel(), 300, 0.01)
    reqs = serve.poisson_requests(pool, 16, rate=300.0, seed=4, lo_log2=16, hi_log2=20, ps=(64, 256))
    alone = serve.Server(slots=1, model=m, train=False).run(reqs, realtime=False)
    mix = serve.Server(slots=4, model=m, train=False).run(reqs, realtime=True)
    for a, b in zip(alone.completions, mix.completions):
        assert a.proposal is not None and b.proposal is not None
        assert torch.equal(a.proposal, b.proposal)
        _same(a, b)
        _check_contract(b)
    # one request against the oracle with its recorded proposal
    c = mix.completions[3]
    r = reqs[3]
    kh = r.keys.cpu().numpy().view(np.uint64)
    ref = oracle.hss(kh, r.p, r.eps, r.seed, sort=False, proposal=c.proposal.cpu().numpy().view(np.uint64))
    assert c.rounds == ref.rounds
    assert np.array_equal(c.offsets.cpu().numpy().astype(np.uint64), ref.offsets)


def test_admission_by_memory_budget(mods):
    hss, serve = mods
    pool = _pool(1, 1 << 20, 60)
    reqs = serve.poisson_requests(pool, 12, rate=1000.0, seed=5, lo_log2=16, hi_log2=20, ps=(64,))
    need = [serve.Server.request_bytes(r.keys.numel(), r.p, nprop=(r.p - 1) * 16) for r in reqs]
    budget = int(1.2 * max(need))
    srv = serve.Server(slots=4, hbm_budget=budget)
    st = srv.run(reqs, realtime=True)
    assert st.max_bytes_in_flight <= budget
    assert all(c.error is None for c in st.completions)
    # a request larger than the whole budget is refused, not queued forever
    big = serve.Request(rid=99, arrival=0.0, keys=pool[0], p=64, eps=0.02, seed=1)
    st2 = serve.Server(slots=2, hbm_budget=budget // 4).run([big], realtime=False)
    assert st2.completions[0].error is not None


def test_online_training_saves_rounds(mods):
    hss, serve = mods
    pool = _pool(3, 1 << 22, 70)
    m = hss.CDFModel().init(3, "log", 1, (1 << 63) - 1)
    reqs = serve.poisson_requests(pool, 80, rate=200.0, seed=6, lo_log2=19, hi_log2=22, ps=(16, 32))
    srv = serve.Server(slots=3, model=m, train=True, train_steps=150)
    srv.warmup()
    st = srv.run(reqs, realtime=True)
    heldout = list(srv.trainer.heldout)
    srv.close()
    s = st.summary()
    print(s, "held-out errors", heldout)
    assert s["completed"] == 80
    for c in st.completions:
        _check_contract(c)
    assert s["served_with_proposal"] >= 20
    assert s["mean_rounds_with_proposal"] < s["mean_rounds_plain"]
    # replay three requests alone with their recorded proposals
    for c in [c for c in st.completions if c.proposal is not None][:3]:
        r = reqs[c.rid]
        res, _ = hss.partition_with_proposal(r.keys, r.p, r.eps, r.seed, c.proposal)
        assert res.rounds == c.rounds
        assert torch.equal(res.offsets, c.offsets) and torch.equal(res.splitters[:r.p - 1], c.splitters[:r.p - 1])


def test_admission_by_free_device_memory(mods):
    """hbm_budget="free": admission reads the device's free memory
    (cudaMemGetInfo plus what the caching allocator holds unused) and keeps
    hbm_reserve free.  With the reserve set so that only some 64 MiB remain,
    small requests are served (their results as alone) and one whose
    workspace needs more is refused rather than queued forever."""
    hss, serve = mods
    pool = _pool(1, 1 << 24, 61)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    reclaim = torch.cuda.memory_reserved() - torch.cuda.memory_allocated()
    reserve = int(free + reclaim) - (64 << 20)
    small = serve.poisson_requests(pool, 6, rate=1000.0, seed=7, lo_log2=14, hi_log2=16, ps=(16,))
    srv = serve.Server(slots=2, hbm_budget="free", hbm_reserve=reserve)
    st = srv.run(small, realtime=False)
    assert all(c.error is None for c in st.completions)
    for c, r in zip(st.completions, sorted(small, key=lambda q: q.rid)):
        kh = r.keys.cpu().numpy().view(np.uint64)
        ref = oracle.hss(kh, r.p, r.eps, r.seed, sort=False)
        assert np.array_equal(c.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    big = serve.Request(rid=99, arrival=0.0, keys=pool[0], p=64, eps=0.02, seed=1)
    assert serve.Server.request_bytes(pool[0].numel(), 64) > (64 << 20)
    st2 = serve.Server(slots=2, hbm_budget="free", hbm_reserve=reserve).run([big], realtime=False)
    assert st2.completions[0].error is not None and st2.completions[0].status == hss.ERR_WORKSPACE
