"""Parity of the batched entry points (hss_sort_batch, hss_partition_batch):
every job of a batch must come out exactly as the oracle computes that job
alone with seed + j -- round counts, sample sizes, |gamma|, unresolved
counts, splitters, offsets, sorted keys and payloads -- and as the single
GPU call computes it."""
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


GENS = [inputs.uniform, inputs.zipf, inputs.gauss_mix, inputs.nested_clusters, inputs.allzeros]


def _jobs(sizes, seed):
    out = []
    for j, n in enumerate(sizes):
        g = GENS[j % len(GENS)]
        out.append(g(n, seed + j) if g is not inputs.allzeros else g(n))
    return out


def _check_job(res, j, keys_j, p, eps, seed, pay_j=None, sorted_out=True, key_type="u64"):
    ref = oracle.hss(keys_j, p, eps, seed, payload=pay_j, sort=sorted_out)
    assert res.job_status[j] == ref.status
    assert res.job_rounds[j] == ref.rounds
    assert res.job_sample_size[j] == [int(x) for x in ref.sample_size]
    assert res.job_gamma[j] == [int(x) for x in ref.gamma]
    assert res.job_unresolved[j] == [int(x) for x in ref.unresolved]
    assert res.job_tol[j] == ref.tol
    assert np.array_equal(res.job_offsets(j).cpu().numpy().astype(np.uint64), ref.offsets)
    from paper_1803_01237_gb300 import hss as h
    k, s, sp = h.cuts_to_numpy(res.job_splitters(j)) if p > 1 else (np.zeros(0), np.zeros(0), np.zeros(0))
    if p > 1:
        want = ref.splitter_key.view(np.uint64) if ref.splitter_key.dtype == np.int64 else ref.splitter_key
        assert np.array_equal(k.view(np.uint64), want)
        assert np.array_equal(s, ref.splitter_seg)
        assert np.array_equal(sp, ref.splitter_spos)
    return ref


@pytest.mark.parametrize("payload", [False, True])
def test_sort_batch_matches_oracle_per_job(hss, payload):
    sizes = [1000, 50000, 1, 7, 200003, 65536, 3000, 120000, 16384, 99991, 0, 40000]
    ps = [4, 16, 1, 7, 13, 4, 1, 64, 4, 9, 1, 3]
    eps, seed = 0.05, 11
    jobs = _jobs(sizes, 100)
    keys = np.concatenate(jobs)
    pay = (np.arange(keys.shape[0], dtype=np.uint64) % (1 << 32)).astype(np.uint32) if payload else None
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(pay.view(np.int32)).cuda() if payload else None
    res = hss.sort_batch(dk, sizes, ps, eps, seed, payload=dp)
    assert res.status == 0
    out = res.keys.cpu().numpy().view(np.uint64)
    outp = res.payload.cpu().numpy().view(np.uint32) if payload else None
    o = 0
    for j, (n, p) in enumerate(zip(sizes, ps)):
        pj = pay[o:o + n] if payload else None
        ref = _check_job(res, j, jobs[j], p, eps, seed + j, pay_j=pj)
        assert np.array_equal(out[o:o + n], ref.out_keys)
        if payload:
            assert np.array_equal(outp[o:o + n], ref.out_payload)
        o += n


def test_partition_batch_matches_single_calls(hss):
    sizes = [70000, 5000, 123457, 30000]
    ps = [32, 5, 100, 2]
    eps, seed = 0.02, 3
    jobs = _jobs(sizes, 7)
    keys = np.concatenate(jobs)
    res = hss.partition_batch(torch.from_numpy(keys.view(np.int64)).cuda(), sizes, ps, eps, seed)
    assert res.status == 0
    for j in range(len(sizes)):
        single, _ = hss.partition(torch.from_numpy(jobs[j].view(np.int64)).cuda(), ps[j], eps, seed + j)
        assert res.job_rounds[j] == single.rounds
        assert res.job_sample_size[j] == single.sample_size
        assert torch.equal(res.job_offsets(j), single.offsets)
        assert torch.equal(res.job_splitters(j), single.splitters[:ps[j] - 1])
        _check_job(res, j, jobs[j], ps[j], eps, seed + j, sorted_out=False)


def test_sort_batch_signed_keys(hss):
    sizes = [3001, 40000, 777]
    ps = [3, 8, 2]
    eps, seed = 0.05, 21
    jobs = [inputs.uniform(n, 50 + j).view(np.int64) for j, n in enumerate(sizes)]
    keys = np.concatenate(jobs)
    res = hss.sort_batch(torch.from_numpy(keys).cuda(), sizes, ps, eps, seed, key_type="i64")
    out = res.keys.cpu().numpy()
    o = 0
    for j, n in enumerate(sizes):
        ref = _check_job(res, j, jobs[j], ps[j], eps, seed + j, key_type="i64")
        assert np.array_equal(out[o:o + n], ref.out_keys)
        o += n


def test_batch_round_limit_is_per_job(hss):
    """A job that needs more rounds than max_rounds reports the limit; the
    other jobs of the batch finish normally."""
    sizes = [1 << 16, 1 << 12]
    ps = [256, 2]
    eps, seed = 0.002, 5
    jobs = [inputs.uniform(sizes[0], 1), inputs.uniform(sizes[1], 2)]
    keys = np.concatenate(jobs)
    res = hss.sort_batch(torch.from_numpy(keys.view(np.int64)).cuda(), sizes, ps, eps, seed, max_rounds=1)
    ref0 = oracle.hss(jobs[0], ps[0], eps, seed, max_rounds=1)
    ref1 = oracle.hss(jobs[1], ps[1], eps, seed + 1, max_rounds=1)
    assert res.job_status[0] == ref0.status and res.job_status[1] == ref1.status
    assert ref0.status == -3
    assert res.status == -3
    assert np.array_equal(res.job_offsets(0).cpu().numpy().astype(np.uint64), ref0.offsets)
    assert np.array_equal(res.job_offsets(1).cpu().numpy().astype(np.uint64), ref1.offsets)
    out = res.keys.cpu().numpy().view(np.uint64)
    assert np.array_equal(out[:sizes[0]], ref0.out_keys) and np.array_equal(out[sizes[0]:], ref1.out_keys)


def test_many_small_jobs(hss):
    """Hundreds of jobs in one call, sizes log-uniform as in the batch
    workload (scaled down), p = max(4, n / 2^14) capped by n."""
    jobs_l, kinds = inputs.batch_jobs(300, 9, lo_log2=6, hi_log2=17)
    sizes = [len(x) for x in jobs_l]
    ps = [max(1, min(n, max(4, n >> 14))) for n in sizes]
    keys = np.concatenate(jobs_l)
    eps, seed = 0.05, 1
    res = hss.sort_batch(torch.from_numpy(keys).cuda(), sizes, ps, eps, seed, key_type="i64")
    assert res.status == 0
    out = res.keys.cpu().numpy()
    o = 0
    for j, n in enumerate(sizes):
        assert np.array_equal(out[o:o + n], np.sort(keys[o:o + n], kind="stable"))
        o += n
    for j in (0, 17, 123, 299):  # full parity on a sample of the jobs
        _check_job(res, j, jobs_l[j], ps[j], eps, seed + j, key_type="i64")


def test_batch_seeds_give_each_job_its_own_call(hss):
    """hss_partition_batch_seeded: job j with seed s_j equals hss_partition
    alone with s_j."""
    sizes = [5000, 70000, 1, 33333]
    ps = [4, 64, 1, 16]
    seeds = [91, 7, 123456789012345, 3]
    keys = np.concatenate([inputs.lognormal_job(n, 9 + j) for j, n in enumerate(sizes)])
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    res = hss.partition_batch(dk, sizes, ps, 0.03, 0, seeds=seeds)
    o = 0
    for j, (n, p, sd) in enumerate(zip(sizes, ps, seeds)):
        one, _ = hss.partition(dk[o:o + n], p, 0.03, sd)
        assert res.job_rounds[j] == one.rounds
        assert torch.equal(res.job_offsets(j), one.offsets)
        if p > 1:
            assert torch.equal(res.job_splitters(j), one.splitters)
        o += n
