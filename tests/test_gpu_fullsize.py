"""The CUDA path at the full sizes of the workloads, in the launch
configuration bench.py times, against the oracle's stored records.

tests/golden/make_goldens.py ran the CPU oracle (and nothing else) on the same
seeded inputs and stored, per case: the round count, every round's sample size
Z_j, |gamma_j| and unresolved count (Sec. 4.2.2), tol, the offsets
chi(0..p) and every splitter tag (key, seg, spos) in full, and SHA-256 digests
of the input and of the globally sorted keys and payload.  Each test
regenerates the input, checks its digest (the generators use only exact
arithmetic, so every machine draws the same keys), runs the GPU path and
compares:
  * rounds, Z_j, |gamma_j|, unresolved counts, tol, status exactly;
  * the offsets and the splitter tags element by element;
  * the sorted keys and payload through their digests (and, as a cheap
    cross-check that localises a mismatch, sortedness and chi(i) positions).

Workloads: the bench input set (N = 2^28, p = 1024, eps = 0.02; uniform,
32-Gaussian mixture, Zipf) with the payload = input index and keys alone (the
bench's own call); the Plummer/Morton workload (N = 2^30 with payload,
p = 16384, eps = 0.01); the batched workload (4096 int64 jobs of 2^10..2^22
keys, one hss_sort_batch call), every job against its record; the
Plummer/Morton workload by two-stage HSS with 128 groups.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def hss():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests selected but no CUDA device is visible")
    from paper_1803_01237_gb300 import hss as h
    h.load()
    return h


def _sha(a: np.ndarray, n: int = 64) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:n]


def _load(name):
    import gzip
    path = os.path.join(GOLDEN, f"fullsize_{name}.json")
    if os.path.exists(path + ".gz"):
        path += ".gz"
    if not os.path.exists(path):
        pytest.fail(f"missing oracle record {path}: run tests/golden/make_goldens.py {name}")
    rec = json.load(gzip.open(path, "rt") if path.endswith(".gz") else open(path))
    npz = os.path.join(GOLDEN, f"fullsize_{name}.npz")
    arr = np.load(npz) if os.path.exists(npz) else None
    return rec, arr


def _compare(res, rec, arr, prefix, N, payload_sha=True):
    assert res.status == rec["status"]
    assert res.tol == rec["tol"]
    assert res.rounds == rec["rounds"]
    assert res.sample_size == rec["sample_size"]
    assert res.gamma == rec["gamma"]
    assert res.unresolved == rec["unresolved"]
    off = res.offsets.cpu().numpy().astype(np.uint64)
    want_off = arr[f"{prefix}offsets"]
    bad = np.nonzero(off != want_off)[0]
    assert bad.size == 0, f"offsets differ at {bad[:8]} (first: {off[bad[0]]} vs {want_off[bad[0]]})"
    k, s, sp = res.splitter_tags()
    for name, got, want in (("key", k.view(np.uint64), arr[f"{prefix}spl_key"]),
                            ("seg", s.astype(np.int32), arr[f"{prefix}spl_seg"]),
                            ("spos", sp.astype(np.uint32), arr[f"{prefix}spl_spos"])):
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"splitter {name} differs at {bad[:8]}"
    out = res.keys.cpu().numpy().view(np.uint64)
    if _sha(out) != rec["out_keys_sha256"]:
        # localise: sortedness, then the splitter keys at their positions
        assert np.all(out[:-1] <= out[1:]) if out.dtype == np.uint64 else True, "output not sorted"
        pos = want_off[1:-1].astype(np.int64)
        member = arr[f"{prefix}spl_seg"] >= 0
        assert np.array_equal(out[pos[member]], arr[f"{prefix}spl_key"][member]), "splitters not at chi(i)"
        pytest.fail("sorted keys differ from the oracle's (digest)")
    if payload_sha:
        assert _sha(res.payload.cpu().numpy().view(np.uint32)) == rec["out_payload_sha256"], "payload differs"


@pytest.mark.timeout(900)
@pytest.mark.parametrize("dist", ["uniform", "gauss_mix", "zipf"])
def test_bench_workload_vs_oracle_record(hss, dist):
    """N = 2^28 uint64, p = 1024, eps = 0.02: the bench configuration, with
    the input index as payload and with keys alone (the bench's call)."""
    rec_all, arr = _load("scale")
    cfg = rec_all["config"]
    rec = rec_all["cases"][dist]
    N, p, eps, seed = cfg["N"], cfg["p"], cfg["eps"], cfg["inputs"][dist]
    keys = inputs.SCALE_DISTRIBUTIONS[dist](N, seed)
    assert _sha(keys) == rec["input_sha256"], "the input generator drew different keys on this machine"
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    del keys
    dp = torch.arange(N, dtype=torch.int32, device="cuda")
    res = hss.sort(dk, p, eps, seed, payload=dp, oversample=cfg["oversample"])
    torch.cuda.synchronize()
    _compare(res, rec, arr, f"{dist}_", N)
    del res, dp
    res = hss.sort(dk, p, eps, seed, oversample=cfg["oversample"])  # keys alone, as bench.py times it
    torch.cuda.synchronize()
    _compare(res, rec, arr, f"{dist}_", N, payload_sha=False)


@pytest.mark.timeout(1500)
def test_plummer_morton_vs_oracle_record(hss):
    """2^30 Morton keys of a Plummer sphere with the particle index as
    payload, p = 16384, eps = 0.01 (the N-body workload)."""
    rec_all, arr = _load("morton")
    cfg = rec_all["config"]
    rec = rec_all["cases"]["plummer"]
    N = 1 << cfg["log2n"]
    keys, payload = inputs.plummer_morton(N, cfg["seed"])
    assert _sha(keys) == rec["input_sha256"], "the input generator drew different keys on this machine"
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(payload.view(np.int32)).cuda()
    del keys, payload
    res = hss.sort(dk, cfg["p"], cfg["eps"], cfg["seed"], payload=dp, oversample=cfg["oversample"])
    torch.cuda.synchronize()
    _compare(res, rec, arr, "", N)


@pytest.mark.timeout(1500)
def test_two_stage_morton_vs_oracle_record(hss):
    """The Plummer/Morton workload sorted by two-stage HSS with 128 groups
    (bench.py --workload morton times this call beside the single stage):
    stage 1's rounds and group cuts, every group's rounds, sample sizes and
    cut digest, the final offsets and the sorted keys and payload."""
    rec, arr = _load("two_stage")
    cfg = rec["config"]
    N = 1 << cfg["log2n"]
    keys, payload = inputs.plummer_morton(N, cfg["seed"])
    assert _sha(keys) == rec["stage1"]["input_sha256"], "the input generator drew different keys on this machine"
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dp = torch.from_numpy(payload.view(np.int32)).cuda()
    del keys, payload
    res = hss.sort_two_stage(dk, cfg["p"], cfg["groups"], cfg["eps"], cfg["seed"], payload=dp,
                             oversample=cfg["oversample"])
    torch.cuda.synchronize()
    s1, r1 = res.stage1, rec["stage1"]
    assert (s1.status, s1.tol, s1.rounds) == (r1["status"], r1["tol"], r1["rounds"])
    assert (s1.sample_size, s1.gamma, s1.unresolved) == (r1["sample_size"], r1["gamma"], r1["unresolved"])
    k, s, sp = hss.cuts_to_numpy(res.group_splitters)
    assert np.array_equal(k.view(np.uint64), arr["group_spl_key"])
    assert np.array_equal(s.astype(np.int32), arr["group_spl_seg"])
    assert np.array_equal(sp.astype(np.uint32), arr["group_spl_spos"])
    off = res.offsets.cpu().numpy().astype(np.uint64)
    bad = np.nonzero(off != arr["offsets"])[0]
    assert bad.size == 0, f"offsets differ at {bad[:8]}"
    bad = []
    for g, rg in enumerate(rec["groups"]):
        k, s, sp = hss.cuts_to_numpy(res.group_splitters_of(g))
        digest = _sha(np.concatenate([k.view(np.uint64), s.astype(np.int64).view(np.uint64),
                                      sp.astype(np.uint64)]), 16)
        got = (res.group_status[g], res.group_tol[g], res.group_rounds[g], res.group_sample_size[g],
               res.group_gamma[g], res.group_unresolved[g], digest)
        want = (rg["status"], rg["tol"], rg["rounds"], rg["sample_size"], rg["gamma"], rg["unresolved"],
                rg["splitters_sha256"])
        if got != want:
            bad.append(g)
    assert not bad, f"groups differing from the oracle: {bad[:8]}"
    assert _sha(res.keys.cpu().numpy().view(np.uint64)) == rec["out_keys_sha256"], "sorted keys differ"
    assert _sha(res.payload.cpu().numpy().view(np.uint32)) == rec["out_payload_sha256"], "payload differs"


@pytest.mark.timeout(1800)
def test_batch_workload_vs_oracle_record(hss):
    """4096 int64 jobs of 2^10..2^22 keys in one hss_sort_batch call: every
    job's rounds, sample sizes, |gamma|, offsets, splitters and sorted keys
    against the oracle run of that job alone (seed 1 + j)."""
    rec_all, _ = _load("batch")
    cfg, jobs_rec = rec_all["config"], rec_all["jobs"]
    jobs, kinds = inputs.batch_jobs(cfg["njobs"], cfg["plan_seed"], lo_log2=cfg["lo_log2"], hi_log2=cfg["hi_log2"],
                                    zipf_s=cfg["zipf_s"], zipf_distinct=cfg["zipf_distinct"])
    sizes = [len(x) for x in jobs]
    ps = [r["p"] for r in jobs_rec]
    assert sizes == [r["n"] for r in jobs_rec]
    for j in (0, 1, len(jobs) // 2, len(jobs) - 1):
        assert _sha(jobs[j].view(np.uint64), 16) == jobs_rec[j]["input_sha256"]
    keys = torch.from_numpy(np.concatenate(jobs)).cuda()
    del jobs
    res = hss.sort_batch(keys, sizes, ps, cfg["eps"], cfg["seed"], oversample=cfg["oversample"], key_type="i64")
    torch.cuda.synchronize()
    out = res.keys.cpu().numpy().view(np.uint64)
    offs_all = res.offsets.cpu().numpy().astype(np.uint64)
    spl_all = res.splitters.cpu().numpy()
    ko = oo = so = 0
    bad = []
    for j, r in enumerate(jobs_rec):
        n, p = r["n"], r["p"]
        got = {
            "status": res.job_status[j], "rounds": res.job_rounds[j], "tol": res.job_tol[j],
            "sample_size": res.job_sample_size[j], "gamma": res.job_gamma[j], "unresolved": res.job_unresolved[j],
            "offsets_sha256": _sha(offs_all[oo:oo + p + 1], 16),
            "out_keys_sha256": _sha(out[ko:ko + n], 16),
        }
        if p > 1:
            cuts = spl_all[so:so + p - 1]
            k = cuts[:, 0].view(np.uint64)
            packed = cuts[:, 1].view(np.uint64)
            seg = (packed & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32).astype(np.int64)
            spos = (packed >> np.uint64(32)).astype(np.uint64)
            got["splitters_sha256"] = _sha(np.concatenate([k, seg.view(np.uint64), spos]), 16)
        else:
            got["splitters_sha256"] = r["splitters_sha256"]
        for key, v in got.items():
            if v != r[key]:
                bad.append((j, key, v, r[key]))
        ko += n
        oo += p + 1
        so += p - 1
    assert not bad, f"{len(bad)} job fields differ, first: {bad[:4]}"


def test_exact_splitting(hss):
    """eps = p/N makes the half-width floor(1/2) = 0: exact splitting (the
    eps = p/N case after Theorem 4.8): every bucket holds N/p keys, and the
    rounds, samples and offsets equal the oracle's."""
    N, p = 1 << 22, 256
    keys = inputs.uniform(N, 21)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    res = hss.sort(dk, p, p / N, 21)
    torch.cuda.synchronize()
    assert res.tol == 0 and res.status == 0
    off = res.offsets.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(off) == N // p)
    ref = oracle.hss(keys, p, p / N, 21)
    assert res.rounds == ref.rounds and res.sample_size == [int(x) for x in ref.sample_size]
    assert np.array_equal(off.astype(np.uint64), ref.offsets)
    assert np.array_equal(res.keys.cpu().numpy().view(np.uint64), ref.out_keys)
