"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work throughout, so every comparison is bit-exact: the sampling
words, the locally sorted segments, the probe ranks, the splitters, the
offsets, the per-round sample sizes and |gamma|, and the sorted output.
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


def host_u64(t):
    return t.cpu().numpy().view(np.uint64)


GENS = {
    "uniform": inputs.uniform,
    "gauss_mix": inputs.gauss_mix,
    "zipf": inputs.zipf,
    "skew1": inputs.skew1,
    "skew2": inputs.skew2,
    "skew3": inputs.skew3,
    "gauss": inputs.gauss,
    "allzeros": inputs.allzeros,
    "nested": inputs.nested_clusters,
    "morton": lambda n, seed: inputs.plummer_morton(n, seed)[0],
}


# ---------------------------------------------------------------------------
# K2: Philox words
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,seg,rnd,spos0", [(1, 0, 1, 0), (0xDEADBEEFCAFEF00D, 1023, 7, 12345),
                                                (2**64 - 1, 65535, 64, 2**31 - 7)])
def test_sample_words_match_oracle(hss, seed, seg, rnd, spos0):
    n = 257
    got = hss.sample_words(seed, seg, rnd, spos0, n).cpu().numpy().view(np.uint64)
    want = np.array([oracle.sample_draw(seed, seg, spos0 + i, rnd) for i in range(n)], dtype=np.uint64)
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# a2: local sort
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,p", [(1000, 1), (50000, 7), (1 << 16, 4), (100003, 3), (200000, 2), (40000, 1),
                                 (16384 * 2, 2), (16385 * 2, 2), (5, 8), (0, 3)])
@pytest.mark.parametrize("gen", ["uniform", "zipf", "skew2", "allzeros", "morton"])
def test_local_sort_matches_oracle(hss, N, p, gen):
    keys = GENS[gen](N, 3)
    pay = (np.arange(N, dtype=np.uint32) * np.uint32(2654435761)).astype(np.uint32)
    if N == 0:
        out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
        assert out.numel() == 0 and outp.numel() == 0
        return
    out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
    want, wantp = oracle.segment_sort(keys, p, payload=pay)
    assert np.array_equal(host_u64(out), want)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), wantp)


@pytest.mark.parametrize("N,p", [(1 << 20, 4), (1 << 20, 1), (1 << 21, 1), (300001, 1), (5 << 17, 5), (70001, 3)])
@pytest.mark.parametrize("gen", list(GENS))
def test_local_sort_keys_only_matches_oracle(hss, N, p, gen):
    """Keys alone take their own kernels (the split hands out slots inside a
    digit with one atomic per key; on-chip sub-buckets are sorted in
    registers): sub-buckets of about 1K, 4K and 8K keys reach all three
    on-chip classes, and skewed inputs reach the fallbacks."""
    keys = GENS[gen](N, 17)
    out = hss.local_sort(dev(keys), p)
    assert np.array_equal(host_u64(out), oracle.segment_sort(keys, p))


@pytest.mark.parametrize("N,p", [(1 << 20, 256), (1 << 22, 4096), (1 << 20, 1024), (3 << 18, 500), (1 << 21, 1)])
@pytest.mark.parametrize("sigma", [2.0, 4.0])
def test_local_sort_keys_only_lognormal(hss, N, p, sigma):
    """Lognormal keys (many binary orders of magnitude) in segments that go
    on chip directly crowd the low groups of a linear digit; the on-chip sort
    then counts again on a logarithmic digit.  Same result as the oracle."""
    keys = inputs.lognormal_job(N, 31, sigma=sigma)
    out = hss.local_sort(dev(keys), p)
    assert np.array_equal(host_u64(out), oracle.segment_sort(keys, p))


@pytest.mark.parametrize("N,p,nvals,share,adjacent", [
    (1 << 20, 2, 3, 0.85, False), (1 << 20, 1, 100, 0.99, False), (600000, 3, 4, 0.5, True),
    (1 << 19, 1, 40, 0.95, False)])
def test_local_sort_keys_only_duplicate_groups(hss, N, p, nvals, share, adjacent):
    keys = inputs.duplicate_groups(N, 19, nvals, share, adjacent)
    out = hss.local_sort(dev(keys), p)
    assert np.array_equal(host_u64(out), oracle.segment_sort(keys, p))


@pytest.mark.parametrize("N,p", [(1 << 18, 1), (300001, 2)])
def test_local_sort_deep_recursion_payload(hss, N, p):
    """Three levels of digit splits: the second level's small buckets are
    sorted on chip in place in the output buffer, payload included."""
    keys = inputs.nested_clusters(N, 11)
    pay = (np.arange(N, dtype=np.uint32) * np.uint32(2654435761)).astype(np.uint32)
    out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
    want, wantp = oracle.segment_sort(keys, p, payload=pay)
    assert np.array_equal(host_u64(out), want)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), wantp)


def _byte_ladder(seed: int, heavy: int, pair: bool):
    """A heavy key value (or two adjacent ones) with a few outliers that
    differ from it in the top bit of each byte: the byte split peels off one
    outlier per level and reaches the heavy values only after eight levels,
    then copies them in a ninth."""
    g = np.random.default_rng(seed)
    v = np.uint64(g.integers(0, 1 << 63, dtype=np.uint64)) | np.uint64(1)
    parts = [np.full(heavy, v, dtype=np.uint64)]
    if pair:
        parts.append(np.full(heavy, v - np.uint64(1), dtype=np.uint64))
    for k in range(8):
        parts.append(np.full(3, v ^ np.uint64(1 << (8 * k + 7)), dtype=np.uint64))
    keys = np.concatenate(parts)
    return keys[g.permutation(keys.size)]


@pytest.mark.parametrize("heavy,pair,p", [(6000, False, 1), (20000, False, 1), (20000, True, 1), (9000, True, 2)])
def test_local_sort_byte_ladder_depth(hss, heavy, pair, p):
    keys = np.concatenate([_byte_ladder(5 + s, heavy, pair) for s in range(p)])
    out = hss.local_sort(dev(keys), p)
    assert np.array_equal(host_u64(out), oracle.segment_sort(keys, p))
    pay = (np.arange(keys.size, dtype=np.uint32) * np.uint32(2654435761)).astype(np.uint32)
    out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
    want, wantp = oracle.segment_sort(keys, p, payload=pay)
    assert np.array_equal(host_u64(out), want)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), wantp)


@pytest.mark.parametrize("N,p", [(1 << 18, 1), (1 << 18, 4), (1 << 20, 16), (300007, 5)])
def test_local_sort_crowded_groups(hss, N, p):
    """Morton keys of a Plummer sphere: the dense core crowds the on-chip
    sort's 10-bit groups, which the largest class re-splits on chip (a
    second counting pass over each crowded group's own range)."""
    keys, _ = inputs.plummer_morton(N, 13)
    pay = (np.arange(N, dtype=np.uint32) * np.uint32(2654435761)).astype(np.uint32)
    out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
    want, wantp = oracle.segment_sort(keys, p, payload=pay)
    assert np.array_equal(host_u64(out), want)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), wantp)
    out2 = hss.local_sort(dev(keys), p)
    out2 = out2[0] if isinstance(out2, tuple) else out2
    assert np.array_equal(host_u64(out2), want)


@pytest.mark.parametrize("N,p,nvals,share,adjacent", [
    (14000, 1, 3, 0.85, False),    # big groups of one value each, many small groups
    (14000, 1, 100, 0.99, False),  # more big groups than the on-chip table holds
    (1500, 1, 2, 0.8, False),      # the smallest on-chip class
    (4000, 1, 4, 0.5, True),       # adjacent values share a group: distinct keys in a big group
    (42001, 3, 5, 0.9, False),     # three segments, each split once first
    (300000, 2, 40, 0.95, False),  # the bench shape in small: split, then on-chip buckets of few values
])
def test_local_sort_duplicate_groups(hss, N, p, nvals, share, adjacent):
    keys = inputs.duplicate_groups(N, 13, nvals, share, adjacent)
    pay = (np.arange(N, dtype=np.uint32) * np.uint32(2654435761)).astype(np.uint32)
    out, outp = hss.local_sort(dev(keys), p, payload=dev(pay))
    want, wantp = oracle.segment_sort(keys, p, payload=pay)
    assert np.array_equal(host_u64(out), want)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), wantp)


@pytest.mark.parametrize("N,p", [(30000, 3), (120000, 2)])
def test_local_sort_signed(hss, N, p):
    keys = inputs.uniform(N, 9).view(np.int64)
    out = hss.local_sort(dev(keys), p, key_type="i64")
    want = oracle.segment_sort(keys, p)
    assert np.array_equal(out.cpu().numpy(), want)


def test_local_sort_in_place(hss):
    N, p = 70000, 2
    keys = inputs.uniform(N, 4)
    d = dev(keys)
    hss.local_sort(d, p, out=d)
    assert np.array_equal(host_u64(d), oracle.segment_sort(keys, p))


# ---------------------------------------------------------------------------
# a5: histogram (ranks of cuts)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gen", ["uniform", "skew2", "allzeros"])
def test_rank_cuts_match_oracle(hss, gen):
    N, p = 6000, 9
    keys = GENS[gen](N, 5)
    srt = oracle.segment_sort(keys, p)
    b = oracle.segment_bounds(N, p)
    g = np.random.default_rng(1)
    ks, ss, ps, want = [], [], [], []
    for _ in range(40):
        s = int(g.integers(0, p)); sp = int(g.integers(0, int(b[s + 1] - b[s])))
        key = int(srt[int(b[s]) + sp])
        ks.append(key); ss.append(s); ps.append(sp)
        want.append(oracle.cut_rank(keys, p, key, seg=s, spos=sp, member=True))
    for key in [0, 7, int(keys.max())]:
        ks.append(key); ss.append(-1); ps.append(0)
        want.append(oracle.cut_rank(keys, p, key, member=False))
    ks += [0, 0]; ss += [-2, -3]; ps += [0, 0]; want += [0, N]
    cuts = hss.cuts_from_numpy(np.array(ks, dtype=np.uint64), ss, ps, "cuda")
    ranks, seg_pos = hss.rank_cuts(dev(srt), p, cuts, want_seg_pos=True)
    assert list(ranks.cpu().numpy()) == want
    assert np.array_equal(seg_pos.cpu().numpy().sum(axis=0), np.array(want))


# ---------------------------------------------------------------------------
# a3-a7: partition, bit-exact against the oracle's round-by-round run
# ---------------------------------------------------------------------------
def _cmp_partition(res, ref):
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


@pytest.mark.parametrize("N,p,eps,seed", [(1 << 20, 64, 0.05, 1), (1 << 16, 16, 0.02, 3), (1 << 18, 4, 0.01, 5),
                                          (12345, 100, 0.05, 2), (1000, 999, 0.05, 2), (3, 5, 0.05, 1),
                                          (1, 1, 0.05, 1), (300, 64, 0.01, 1)])
def test_partition_matches_oracle(hss, N, p, eps, seed):
    keys = inputs.uniform(N, seed)
    res, _ = hss.partition(dev(keys), p, eps, seed)
    ref = oracle.hss(keys, p, eps, seed, sort=False)
    _cmp_partition(res, ref)


@pytest.mark.parametrize("gen", ["gauss_mix", "zipf", "skew1", "skew2", "skew3", "gauss", "allzeros"])
def test_partition_distributions(hss, gen):
    N, p, eps, seed = 1 << 17, 32, 0.02, 11
    keys = GENS[gen](N, seed)
    res, _ = hss.partition(dev(keys), p, eps, seed)
    ref = oracle.hss(keys, p, eps, seed, sort=False)
    _cmp_partition(res, ref)


def test_partition_signed(hss):
    N, p, eps, seed = 50000, 10, 0.05, 4
    keys = inputs.uniform(N, 4).view(np.int64)
    res, _ = hss.partition(dev(keys), p, eps, seed, key_type="i64")
    ref = oracle.hss(keys, p, eps, seed, sort=False)
    _cmp_partition(res, ref)


def test_partition_oversample_and_round_limit(hss):
    N, p, eps = 1 << 16, 32, 0.002
    keys = inputs.uniform(N, 2)
    for s in (1.0, 2.5, 20.0):
        res, _ = hss.partition(dev(keys), p, eps, 9, oversample=s)
        ref = oracle.hss(keys, p, eps, 9, oversample=s, sort=False)
        _cmp_partition(res, ref)
    res, _ = hss.partition(dev(keys), p, eps, 9, max_rounds=1, allow_round_limit=True)
    ref = oracle.hss(keys, p, eps, 9, max_rounds=1, sort=False)
    assert res.status == -3 and ref.status == -3
    _cmp_partition(res, ref)


# ---------------------------------------------------------------------------
# a8/a9 and the whole path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,p,eps,seed,payload", [(1 << 20, 64, 0.05, 1, False), (1 << 20, 64, 0.05, 1, True),
                                                  (1 << 18, 4, 0.02, 3, True), (99991, 13, 0.05, 2, True),
                                                  (1000, 999, 0.05, 2, False), (7, 7, 0.05, 1, True),
                                                  (1 << 15, 1, 0.05, 1, True), (0, 4, 0.05, 1, False)])
def test_sort_matches_oracle(hss, N, p, eps, seed, payload):
    keys = inputs.uniform(N, seed)
    pay = np.arange(N, dtype=np.uint32) if payload else None
    res = hss.sort(dev(keys), p, eps, seed, payload=dev(pay) if payload else None)
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    _cmp_partition(res, ref)
    assert np.array_equal(host_u64(res.keys), ref.out_keys)
    if payload:
        assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


@pytest.mark.parametrize("gen", ["gauss_mix", "zipf", "skew2", "allzeros", "skew3", "nested", "morton"])
def test_sort_distributions(hss, gen):
    N, p, eps, seed = 1 << 18, 8, 0.02, 5
    keys = GENS[gen](N, seed)
    pay = np.arange(N, dtype=np.uint32)
    res = hss.sort(dev(keys), p, eps, seed, payload=dev(pay))
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    _cmp_partition(res, ref)
    assert np.array_equal(host_u64(res.keys), ref.out_keys)
    assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


@pytest.mark.parametrize("gen", list(GENS))
def test_sort_keys_only_distributions(hss, gen):
    """The whole path with keys alone (the bench's call) at a size where both
    the local sort and the merge split every segment before the on-chip sorts."""
    N, p, eps, seed = 1 << 21, 8, 0.02, 7
    keys = GENS[gen](N, seed)
    res = hss.sort(dev(keys), p, eps, seed)
    ref = oracle.hss(keys, p, eps, seed)
    _cmp_partition(res, ref)
    assert np.array_equal(host_u64(res.keys), ref.out_keys)


def test_sort_signed(hss):
    N, p, eps, seed = 1 << 17, 3, 0.05, 6
    keys = inputs.uniform(N, 6).view(np.int64)
    res = hss.sort(dev(keys), p, eps, seed, key_type="i64")
    ref = oracle.hss(keys, p, eps, seed)
    assert np.array_equal(res.keys.cpu().numpy(), ref.out_keys)
    _cmp_partition(res, ref)


def test_exchange_and_merge_steps(hss):
    """hss_exchange then hss_merge reproduce the oracle's buckets and output."""
    N, p, eps, seed = 1 << 17, 16, 0.05, 8
    keys = inputs.uniform(N, seed)
    pay = np.arange(N, dtype=np.uint32)
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    srt, srtp = hss.local_sort(dev(keys), p, payload=dev(pay))
    cuts = hss.cuts_from_numpy(ref.splitter_key, ref.splitter_seg, ref.splitter_spos, "cuda")
    ranks, seg_pos = hss.rank_cuts(srt, p, cuts, want_seg_pos=True)
    assert np.array_equal(ranks.cpu().numpy().astype(np.uint64), ref.offsets[1:-1])
    off = torch.from_numpy(ref.offsets.view(np.int64)).cuda()
    bk, bp = hss.exchange(srt, p, seg_pos, off, sorted_payload=srtp)
    # every bucket holds the oracle's bucket as a multiset, runs in segment order
    bkh, refk = host_u64(bk), ref.out_keys
    for b in range(p):
        lo, hi = int(ref.offsets[b]), int(ref.offsets[b + 1])
        assert np.array_equal(np.sort(bkh[lo:hi]), refk[lo:hi])
    out, outp = hss.merge(bk, p, off, bucket_payload=bp)
    assert np.array_equal(host_u64(out), ref.out_keys)
    assert np.array_equal(outp.cpu().numpy().view(np.uint32), ref.out_payload)


def test_sort_host_matches_oracle(hss):
    N, p, eps, seed = 1 << 18, 16, 0.05, 12
    keys = inputs.uniform(N, seed)
    pay = np.arange(N, dtype=np.uint32)
    out, outp, spl, off, st = hss.sort_host(keys, p, eps, seed, payload=pay)
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    assert np.array_equal(out, ref.out_keys)
    assert np.array_equal(outp, ref.out_payload)
    assert np.array_equal(off, ref.offsets)


def test_repeatable_and_launch_count(hss):
    N, p = 1 << 18, 8
    keys = dev(inputs.uniform(N, 1))
    a = hss.launch_count()
    r1 = hss.sort(keys, p, 0.02, 1)
    k1 = r1.keys.clone()
    r2 = hss.sort(keys, p, 0.02, 1)
    assert torch.equal(k1, r2.keys)
    assert hss.launch_count() - a == r1.kernel_launches + r2.kernel_launches > 0


# ---------------------------------------------------------------------------
# Sampling schedules: the k-round schedule of Theorem 4.7 and the
# equal-per-interval (HykSort) sampling, bit-exact against the oracle.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("schedule,k", [("theory", 1), ("theory", 3), ("equal", 0)])
@pytest.mark.parametrize("gen", ["uniform", "gauss_mix", "zipf"])
def test_schedules_match_oracle(hss, schedule, k, gen):
    N, p, eps, seed = 1 << 18, 32, 0.02, 7
    keys = GENS[gen](N, seed)
    res, _ = hss.partition(dev(keys), p, eps, seed, schedule=schedule, schedule_k=k)
    ref = oracle.hss(keys, p, eps, seed, sort=False, schedule=schedule, schedule_k=k)
    _cmp_partition(res, ref)


def test_schedule_sort_output(hss):
    N, p, eps, seed = 200003, 12, 0.01, 3
    keys = inputs.gauss_mix(N, seed)
    pay = np.arange(N, dtype=np.uint32)
    for schedule, k in (("theory", 2), ("equal", 0)):
        res = hss.sort(dev(keys), p, eps, seed, payload=dev(pay), schedule=schedule, schedule_k=k)
        ref = oracle.hss(keys, p, eps, seed, payload=pay, schedule=schedule, schedule_k=k)
        _cmp_partition(res, ref)
        assert np.array_equal(host_u64(res.keys), ref.out_keys)
        assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


# ---------------------------------------------------------------------------
# a5: both histogram forms (probe-side and staged) give the oracle's rounds
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,p,eps,seed", [(1 << 16, 1024, 0.05, 1), (1 << 18, 512, 0.02, 2), (100003, 777, 0.05, 3),
                                          (1 << 20, 64, 0.05, 4), (5000, 4999, 0.05, 5), (3000, 2, 0.01, 6)])
@pytest.mark.parametrize("gen", ["uniform", "zipf", "allzeros"])
@pytest.mark.parametrize("mode", ["probe", "staged"])
def test_histogram_forms_match_oracle(hss, N, p, eps, seed, gen, mode):
    """Forced staged or probe-side histograms, large p against N (segments
    of 1 to 64 keys), duplicates and all-equal keys: same rounds, samples,
    splitters and offsets as the oracle."""
    keys = GENS[gen](N, seed) if gen != "allzeros" else inputs.allzeros(N)
    flags = hss.FLAG_HIST_STAGED if mode == "staged" else hss.FLAG_HIST_PROBE
    res, _ = hss.partition(dev(keys), p, eps, seed, flags=flags)
    ref = oracle.hss(keys, p, eps, seed, sort=False)
    _cmp_partition(res, ref)


def test_histogram_auto_large_p_sort(hss):
    """The automatic choice at large p (staged in round 1) on a sort with payload."""
    N, p, eps, seed = 1 << 19, 2048, 0.02, 8
    keys = inputs.gauss_mix(N, seed)
    pay = np.arange(N, dtype=np.uint32)
    res = hss.sort(dev(keys), p, eps, seed, payload=dev(pay))
    ref = oracle.hss(keys, p, eps, seed, payload=pay)
    _cmp_partition(res, ref)
    assert np.array_equal(host_u64(res.keys), ref.out_keys)
    assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


def test_histogram_staged_with_proposal(hss):
    """The proposal pass (all cuts share the first interval) in staged form."""
    N, p, eps, seed = 1 << 18, 256, 0.02, 9
    keys = inputs.uniform(N, seed)
    srt = np.sort(keys)
    prop = srt[[(i * N) // p + 37 for i in range(1, p)]]
    for flags in (hss.FLAG_HIST_STAGED, hss.FLAG_HIST_PROBE):
        res, _ = hss.partition_with_proposal(dev(keys), p, eps, seed, dev(prop), flags=flags)
        ref = oracle.hss(keys, p, eps, seed, sort=False, proposal=prop)
        _cmp_partition(res, ref)


# ---------------------------------------------------------------------------
# a6: the rounds driven on the device (graph loop) and from the host
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,p,eps,seed,max_rounds", [(1 << 20, 64, 0.05, 1, 0), (1 << 18, 1024, 0.02, 4, 0),
                                                     (1 << 16, 16, 0.001, 3, 2), (5000, 4999, 0.05, 2, 0),
                                                     (1 << 17, 8, 10.0, 1, 0)])
def test_device_and_host_rounds_agree_with_oracle(hss, N, p, eps, seed, max_rounds):
    """The default device-driven loop (one CUDA graph, a device kernel deciding
    each next round) and the host-driven loop give the oracle's rounds, sample
    sizes, |gamma|, unresolved counts, splitters and offsets -- also when the
    round limit stops them (status HSS_ERR_ROUND_LIMIT) and when no round is
    needed (eps >= 1)."""
    keys = inputs.uniform(N, seed)
    ref = oracle.hss(keys, p, eps, seed, sort=False, max_rounds=max_rounds or 64)
    dk = dev(keys)
    for flags in (hss.FLAG_DEVICE_ROUNDS, hss.FLAG_HOST_ROUNDS, 0, 0):  # default: host first, then the graph
        res, _ = hss.partition(dk, p, eps, seed, max_rounds=max_rounds, flags=flags, allow_round_limit=True)
        assert res.status == ref.status
        _cmp_partition(res, ref)


def test_partition_returns_before_the_gpu_and_stats_come_later(hss):
    """Without statistics hss_partition enqueues everything and returns;
    hss_call_stats then reads the rounds, sample sizes and status from the
    workspace, equal to the oracle's."""
    N, p, eps, seed = 1 << 20, 256, 0.02, 9
    keys = inputs.gauss_mix(N, seed)
    dk = dev(keys)
    spl, off, ws = hss.partition_async(dk, p, eps, seed, flags=hss.FLAG_DEVICE_ROUNDS)
    rc, st = hss.call_stats("partition", N, p, eps, seed, ws, flags=hss.FLAG_DEVICE_ROUNDS)
    ref = oracle.hss(keys, p, eps, seed, sort=False)
    assert rc == 0 and st.status == 0
    assert st.rounds == ref.rounds
    assert [int(x) for x in st.sample_size[:st.rounds]] == [int(x) for x in ref.sample_size]
    assert [int(x) for x in st.gamma[:st.rounds]] == [int(x) for x in ref.gamma]
    assert [int(x) for x in st.unresolved[:st.rounds + 1]] == [int(x) for x in ref.unresolved]
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.offsets)
    # a host-driven call leaves the same record
    _, off2, ws2 = hss.partition_async(dk, p, eps, seed, flags=hss.FLAG_HOST_ROUNDS)
    rc2, st2 = hss.call_stats("partition", N, p, eps, seed, ws2, flags=hss.FLAG_HOST_ROUNDS)
    assert rc2 == 0 and st2.rounds == ref.rounds
    assert [int(x) for x in st2.sample_size[:st2.rounds]] == [int(x) for x in ref.sample_size]
