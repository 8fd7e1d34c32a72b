"""Parity of hss_sort_two_stage with the oracle's two-stage HSS: stage 1's
rounds, sample sizes, group cuts and group offsets, every group's stage-2
rounds and cuts, the final offsets and the sorted keys and payloads must be
identical."""
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


GENS = {"uniform": inputs.uniform, "gauss_mix": inputs.gauss_mix, "zipf": inputs.zipf,
        "nested": inputs.nested_clusters, "skew3": inputs.skew3}


def _cuts_equal(h, packed, key, seg, spos):
    k, s, sp = h.cuts_to_numpy(packed)
    want = key.view(np.uint64) if key.dtype == np.int64 else key
    assert np.array_equal(k.view(np.uint64), want)
    assert np.array_equal(s, seg)
    assert np.array_equal(sp, spos)


def _check(h, res, ref, r, p, payload):
    pg = p // r
    s1, t1 = res.stage1, ref.stage1
    assert s1.rounds == t1.rounds
    assert s1.sample_size == [int(x) for x in t1.sample_size]
    assert s1.gamma == [int(x) for x in t1.gamma]
    assert s1.unresolved == [int(x) for x in t1.unresolved]
    assert s1.tol == t1.tol
    _cuts_equal(h, res.group_splitters, t1.splitter_key, t1.splitter_seg, t1.splitter_spos)
    assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
    for g in range(r):
        t2 = ref.stage2[g]
        assert res.group_status[g] == t2.status
        assert res.group_rounds[g] == t2.rounds
        assert res.group_sample_size[g] == [int(x) for x in t2.sample_size]
        assert res.group_tol[g] == t2.tol
        if pg > 1:
            _cuts_equal(h, res.group_splitters_of(g), t2.splitter_key, t2.splitter_seg, t2.splitter_spos)
    out = res.keys.cpu().numpy()
    want = ref.out_keys.view(np.int64) if ref.out_keys.dtype == np.uint64 else ref.out_keys
    assert np.array_equal(out, want)
    if payload is not None:
        assert np.array_equal(res.payload.cpu().numpy().view(np.uint32), ref.out_payload)


@pytest.mark.parametrize("gen", list(GENS))
@pytest.mark.parametrize("N,p,r", [(1 << 18, 64, 8), (300007, 96, 12), (1 << 16, 16, 16)])
def test_two_stage_matches_oracle(hss, gen, N, p, r):
    eps, seed = 0.03, 21
    keys = GENS[gen](N, 4)
    res = hss.sort_two_stage(torch.from_numpy(keys.view(np.int64)).cuda(), p, r, eps, seed)
    ref = oracle.hss_two_stage(keys, p, r, eps, seed)
    assert res.status == 0 and res.groups == r
    _check(hss, res, ref, r, p, None)


@pytest.mark.parametrize("key_type", ["u64", "i64"])
def test_two_stage_payload_and_signed_keys(hss, key_type):
    N, p, r, eps, seed = 200003, 128, 16, 0.02, 5
    keys = inputs.zipf(N, 7)
    if key_type == "i64":
        keys = (keys.view(np.int64) - np.int64(1 << 40)).astype(np.int64)
    payload = (np.arange(N, dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(payload.view(np.int32)).cuda()
    res = hss.sort_two_stage(dk, p, r, eps, seed, payload=dp, key_type=key_type)
    ref = oracle.hss_two_stage(keys, p, r, eps, seed, payload=payload)
    assert res.status == 0
    _check(hss, res, ref, r, p, payload)


@pytest.mark.parametrize("flags", ["host", "device"])
def test_two_stage_round_drivers_agree(hss, flags):
    N, p, r, eps, seed = 1 << 19, 256, 16, 0.02, 8
    keys = inputs.gauss_mix(N, 2)
    f = hss.FLAG_HOST_ROUNDS if flags == "host" else hss.FLAG_DEVICE_ROUNDS
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    ref = oracle.hss_two_stage(keys, p, r, eps, seed)
    for _ in range(2):  # the second call of a shape may run a cached graph
        res = hss.sort_two_stage(dk, p, r, eps, seed, flags=f)
        _check(hss, res, ref, r, p, None)


def test_two_stage_all_equal_keys(hss):
    N, p, r = 1 << 16, 32, 4
    keys = inputs.allzeros(N)
    res = hss.sort_two_stage(torch.from_numpy(keys.view(np.int64)).cuda(), p, r, 0.05, 3)
    ref = oracle.hss_two_stage(keys, p, r, 0.05, 3)
    _check(hss, res, ref, r, p, None)


def test_two_stage_refuses_bad_group_counts(hss):
    keys = torch.zeros(1 << 12, dtype=torch.int64, device="cuda")
    for p, r in [(16, 1), (16, 5), (16, 32)]:
        with pytest.raises(hss.HSSError):
            hss.sort_two_stage(keys, p, r, 0.05, 1)
    with pytest.raises(hss.HSSError):
        hss.sort_two_stage(keys[:40], 32, 4, 0.05, 1)  # fewer than 2p keys


def test_two_stage_round_limit_matches_oracle(hss):
    """With one round per stage the splitters stay unresolved: both stages
    report the round limit, keep the closest cuts seen (Sec. 4.2.2 step 5),
    and the result is still the oracle's, stage by stage."""
    N, p, r, eps, seed = 1 << 18, 64, 8, 0.002, 4
    keys = inputs.gauss_mix(N, 6)
    res = hss.sort_two_stage(torch.from_numpy(keys.view(np.int64)).cuda(), p, r, eps, seed, max_rounds=1)
    ref = oracle.hss_two_stage(keys, p, r, eps, seed, max_rounds=1)
    assert ref.stage1.status == res.stage1.status == hss.ERR_ROUND_LIMIT
    assert res.status == hss.ERR_ROUND_LIMIT
    _check(hss, res, ref, r, p, None)
