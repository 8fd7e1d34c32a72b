"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each pin ties one part of the oracle to a fact fixed by the paper, by the
mathematics, by a published test vector or by an independent library routine
(numpy's stable sort and its own comparisons), so that a dropped term, a wrong
sign or index or a transposed operand in the oracle fails at least one test.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10: the published known-answer vectors (Random123 distribution of
# Salmon et al., SC'11).
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for case in kat["vectors"]:
        ctr = [int(x, 16) for x in case["ctr"]]
        key = [int(x, 16) for x in case["key"]]
        want = [int(x, 16) for x in case["out"]]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(v) for v in got] == want, case


def test_sample_draw_word_pairing():
    # Even and odd positions of a pair take the low and high halves of one block.
    seed, seg, rnd = 0x0123456789ABCDEF, 7, 3
    for spos in (0, 10, 12345):
        x = oracle.philox4x32_10([spos >> 1, seg, rnd, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.sample_draw(seed, seg, spos & ~1, rnd) == (int(x[1]) << 32) | int(x[0])
        assert oracle.sample_draw(seed, seg, spos | 1, rnd) == (int(x[3]) << 32) | int(x[2])


def test_sample_draw_is_uniform():
    # 64-bit words of a good generator: mean of top-16-bit buckets is flat.
    vals = np.array([oracle.sample_draw(1, s, i, 1) for s in range(4) for i in range(4096)], dtype=np.uint64)
    top = (vals >> np.uint64(60)).astype(np.int64)
    counts = np.bincount(top, minlength=16)
    exp = vals.size / 16
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


# ---------------------------------------------------------------------------
# Thresholds and targets (Sec. 2, Sec. 6 "s/delta" sampling)
# ---------------------------------------------------------------------------
def test_threshold_closed_forms():
    assert oracle.threshold(5.0, 64, 640) == (1 << 63, False)          # q = 1/2
    assert oracle.threshold(5.0, 64, 320) == (0, True)                 # q = 1
    assert oracle.threshold(5.0, 64, 100) == (0, True)                 # q > 1 -> take all
    assert oracle.threshold(5.0, 64, 0) == (0, True)
    assert oracle.threshold(1.0, 1, 4) == (1 << 62, False)             # q = 1/4
    T, ta = oracle.threshold(5.0, 1024, 1 << 28)
    assert not ta and T == int(math.floor(5 * 1024 / (1 << 28) * 2 ** 64))


def test_tolerance_closed_forms():
    assert oracle.tolerance(1 << 20, 64, 0.05) == 409          # 2^20*0.05/128 = 409.6
    assert oracle.tolerance(1 << 28, 1024, 0.02) == 2621
    assert oracle.tolerance(1 << 30, 16384, 0.01) == 327
    assert oracle.tolerance(100, 10, 0.1) == 0


# ---------------------------------------------------------------------------
# Local sort with implicit tagging (Sec. 5, Sec. 6.1) against numpy.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 3, 16, 64])
@pytest.mark.parametrize("gen", ["uniform", "skew2", "allzeros", "zipf"])
def test_segment_sort_matches_numpy_stable(p, gen):
    N = 5000
    keys = {"uniform": inputs.uniform, "skew2": inputs.skew2, "allzeros": inputs.allzeros,
            "zipf": lambda n, s: inputs.zipf(n, s, distinct=50)}[gen](N, 11)
    payload = np.arange(N, dtype=np.uint32) * np.uint32(7)
    out, opay = oracle.segment_sort(keys, p, payload=payload)
    b = oracle.segment_bounds(N, p)
    for s in range(p):
        lo, hi = int(b[s]), int(b[s + 1])
        order = np.argsort(keys[lo:hi], kind="stable")
        assert np.array_equal(out[lo:hi], keys[lo:hi][order])
        assert np.array_equal(opay[lo:hi], payload[lo:hi][order])


def test_segment_sort_signed():
    N = 3001
    keys = inputs.uniform(N, 5).view(np.int64)
    out = oracle.segment_sort(keys, 7)
    b = oracle.segment_bounds(N, 7)
    for s in range(7):
        lo, hi = int(b[s]), int(b[s + 1])
        assert np.array_equal(out[lo:hi], np.sort(keys[lo:hi], kind="stable"))


def test_segment_bounds_uneven():
    b = oracle.segment_bounds(10, 4)
    assert list(b) == [0, 2, 5, 7, 10]
    b = oracle.segment_bounds(3, 5)
    assert list(b) == [0, 0, 1, 1, 2, 3]


# ---------------------------------------------------------------------------
# The histogram of one probe (Sec. 3.3 step 2) against brute force.
# ---------------------------------------------------------------------------
def _global_order(keys, p):
    """Brute force: rank of every input element in (key, global index) order."""
    N = keys.shape[0]
    order = np.argsort(keys, kind="stable")
    rank_of = np.empty(N, dtype=np.int64)
    rank_of[order] = np.arange(N)
    return order, rank_of


def _sorted_pos_to_input_index(keys, p):
    """Original input index of (seg, spos) after the stable local sort."""
    b = oracle.segment_bounds(keys.shape[0], p)
    idx = []
    for s in range(p):
        lo, hi = int(b[s]), int(b[s + 1])
        idx.append(lo + np.argsort(keys[lo:hi], kind="stable"))
    return b, idx


@pytest.mark.parametrize("gen", ["uniform", "skew2", "allzeros"])
def test_cut_rank_brute_force(gen):
    N, p = 2000, 9
    keys = {"uniform": inputs.uniform, "skew2": inputs.skew2, "allzeros": inputs.allzeros}[gen](N, 3)
    _, rank_of = _global_order(keys, p)
    b, idx = _sorted_pos_to_input_index(keys, p)
    g = np.random.default_rng(0)
    for _ in range(60):
        s = int(g.integers(0, p))
        n = int(b[s + 1] - b[s])
        spos = int(g.integers(0, n))
        key = int(keys[idx[s][spos]])
        want = int(rank_of[idx[s][spos]])
        assert oracle.cut_rank(keys, p, key, seg=s, spos=spos, member=True) == want
    # non-member cut (k, -1): number of keys strictly smaller than k
    for key in [0, 1, 50, int(keys.max()), int(keys.max()) + 1 if int(keys.max()) < 2**64 - 1 else 0]:
        assert oracle.cut_rank(keys, p, key, member=False) == int((keys < np.uint64(key)).sum())


# ---------------------------------------------------------------------------
# The whole method.
# ---------------------------------------------------------------------------
def _check_result(keys, p, eps, res, payload=None):
    N = keys.shape[0]
    # Sorted output equals numpy's stable sort of the whole input (Sec. 2).
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(res.out_keys, keys[order])
    if payload is not None:
        assert np.array_equal(res.out_payload, payload[order])
    # Offsets: chi(0) = 0, chi(p) = N, monotone, every chi(i) in its target range.
    off = res.offsets.astype(np.int64)
    assert off[0] == 0 and off[-1] == N
    assert np.all(np.diff(off) >= 0)
    tol = oracle.tolerance(N, p, eps)
    assert res.tol == tol
    t = np.array([(i * N) // p for i in range(1, p)], dtype=np.int64)
    if res.status == 0:
        assert np.all(np.abs(off[1:-1] - t) <= tol)
        sizes = np.diff(off)
        assert sizes.max() <= -(-N // p) + 2 * tol
    # Each splitter is the input element of rank chi(i) (S(i) = I(chi(i))).
    _, rank_of = _global_order(keys, p)
    b, idx = _sorted_pos_to_input_index(keys, p)
    for i in range(p - 1):
        seg = int(res.splitter_seg[i])
        if seg >= 0:
            e = idx[seg][int(res.splitter_spos[i])]
            assert int(rank_of[e]) == int(off[i + 1])
            assert keys[e] == res.splitter_key[i]
            assert res.out_keys[int(off[i + 1])] == res.splitter_key[i]
        elif seg == -2:
            assert off[i + 1] == 0
        elif seg == -3:
            assert off[i + 1] == N


@pytest.mark.parametrize("gen", ["uniform", "gauss_mix", "zipf", "skew1", "skew3", "allzeros"])
def test_hss_uniformity_of_contract(gen):
    N, p, eps = 1 << 14, 32, 0.05
    f = {"uniform": inputs.uniform, "gauss_mix": inputs.gauss_mix, "zipf": inputs.zipf,
         "skew1": inputs.skew1, "skew3": inputs.skew3, "allzeros": inputs.allzeros}[gen]
    keys = f(N, 1)
    payload = np.arange(N, dtype=np.uint32)
    res = oracle.hss(keys, p, eps, seed=1, payload=payload)
    assert res.status == 0
    _check_result(keys, p, eps, res, payload)


def test_hss_signed_keys():
    N, p, eps = 9000, 12, 0.1
    keys = inputs.uniform(N, 4).view(np.int64)
    res = oracle.hss(keys, p, eps, seed=9)
    assert res.status == 0
    _check_result(keys, p, eps, res)


def test_hss_ragged_and_tiny():
    for N, p in [(1, 1), (7, 7), (10, 4), (3, 5), (0, 3), (1000, 999), (12345, 100)]:
        keys = inputs.uniform(N, N + p)
        res = oracle.hss(keys, p, 0.05, seed=2)
        assert res.status == 0
        _check_result(keys, p, 0.05, res)


def test_hss_p_equals_one():
    keys = inputs.uniform(1000, 1)
    res = oracle.hss(keys, 1, 0.05, seed=1)
    assert res.rounds == 0 and list(res.offsets) == [0, 1000]
    assert np.array_equal(res.out_keys, np.sort(keys))


def test_hss_allzeros_is_identity_permutation():
    # Sec. 7.5 AllZeros: with (key, processor, index) tags every rank is the
    # global index, so the output is the input order and chi(i) is in range.
    N, p = 4096, 16
    keys = inputs.allzeros(N)
    payload = np.arange(N, dtype=np.uint32)
    res = oracle.hss(keys, p, 0.05, seed=3, payload=payload)
    assert np.array_equal(res.out_payload, payload)


def test_take_all_round_is_exact_selection():
    # When s*p >= |gamma_0| = N the first round samples every key, every t_i
    # is a probe and chi(i) = t_i exactly in one round.
    N, p = 300, 64
    keys = inputs.uniform(N, 8)
    res = oracle.hss(keys, p, 0.01, seed=1, oversample=5.0)
    assert res.rounds == 1 and int(res.sample_size[0]) == N
    t = [(i * N) // p for i in range(1, p)]
    assert list(res.offsets[1:-1]) == t


def test_large_eps_needs_no_round():
    # eps >= p makes the half-width N eps/(2p) >= N/2, so the sentinel ranks 0
    # and N already lie in every target range: no histogramming.
    N, p = 1000, 10
    res = oracle.hss(inputs.uniform(N, 1), p, float(p), seed=1)
    assert res.rounds == 0
    _check_result(inputs.uniform(N, 1), p, float(p), res)
    # just below that, some splitter needs a round
    assert oracle.hss(inputs.uniform(N, 1), p, 0.5 * p, seed=1).rounds >= 1


# ---------------------------------------------------------------------------
# Round-level pins, from the per-round trace.
# ---------------------------------------------------------------------------
def _trace_case(gen="uniform", N=1 << 13, p=16, eps=0.02, seed=5, oversample=5.0):
    keys = {"uniform": inputs.uniform, "zipf": lambda n, s: inputs.zipf(n, s, distinct=300)}[gen](N, seed)
    res = oracle.hss(keys, p, eps, seed=seed, oversample=oversample, trace=True)
    return keys, res


@pytest.mark.parametrize("gen", ["uniform", "zipf"])
def test_histogram_and_update_against_brute_force(gen):
    """L_j(i)/U_j(i) after every round equal the best brute-force-ranked probe
    seen so far below/above t_i (Sec. 4.2.2 step 3)."""
    N, p, eps = 1 << 13, 16, 0.02
    keys, res = _trace_case(gen, N, p, eps)
    assert res.status == 0 and res.rounds >= 2
    _, rank_of = _global_order(keys, p)
    b, idx = _sorted_pos_to_input_index(keys, p)
    t = np.array([(i * N) // p for i in range(1, p)], dtype=np.int64)
    seen = np.zeros(0, dtype=np.int64)
    for r in range(res.rounds):
        smp = res.samples[r]
        # probe tags map back to input elements; their key must match
        ranks = []
        for key, seg, spos in smp:
            e = idx[int(seg)][int(spos)]
            assert keys[e] == key
            ranks.append(int(rank_of[e]))
        ranks = np.array(ranks, dtype=np.int64)
        assert np.all(np.diff(ranks) > 0)  # sorted sample = increasing ranks
        seen = np.concatenate([seen, ranks])
        for i in range(p - 1):
            below = seen[seen <= t[i]]
            above = seen[seen >= t[i]]
            wantL = int(below.max()) if below.size else 0
            wantU = int(above.min()) if above.size else N
            assert int(res.trace_lrank[r + 1, i]) == wantL
            assert int(res.trace_urank[r + 1, i]) == wantU


@pytest.mark.parametrize("gen", ["uniform", "zipf"])
def test_sampling_set_rederived(gen):
    """Round j samples exactly the keys strictly inside unresolved intervals
    whose Philox word is below T_j (Sec. 4.2.1 sampling method)."""
    N, p, eps = 1 << 13, 16, 0.02
    keys, res = _trace_case(gen, N, p, eps)
    b, idx = _sorted_pos_to_input_index(keys, p)
    _, rank_of = _global_order(keys, p)
    # global rank of every (seg, spos)
    rank_sp = [rank_of[idx[s]] for s in range(p)]
    for r in range(res.rounds):
        L = res.trace_lrank[r].astype(np.int64)
        U = res.trace_urank[r].astype(np.int64)
        flags = res.trace_resolved[r]
        resolved = (flags & 1) != 0
        lmem = (flags & 2) != 0
        # region = union over unresolved i of ranks in [L + [L member], U)
        inside = np.zeros(N, dtype=bool)
        gamma = 0
        done = set()
        for i in range(p - 1):
            if resolved[i]:
                continue
            lo = int(L[i]) + int(lmem[i])
            hi = int(U[i])
            if (lo, hi) in done:
                continue
            done.add((lo, hi))
            inside[lo:hi] = True
            gamma += max(hi - lo, 0)
        assert gamma == int(res.gamma[r])
        q = min(1.0, 5.0 * p / gamma)
        take_all = q >= 1.0
        T = 0 if take_all else int(math.floor(math.ldexp(q, 64)))
        want = set()
        for s in range(p):
            for spos in range(len(rank_sp[s])):
                if inside[rank_sp[s][spos]] and (take_all or oracle.sample_draw(5, s, spos, r + 1) < T):
                    want.add((s, spos))
        got = {(int(sg), int(sp)) for _, sg, sp in res.samples[r]}
        assert got == want


def test_intervals_identical_or_disjoint_and_monotone():
    """Splitter intervals are identical or disjoint (Sec. 4.2.2) and L/U only
    improve across rounds (proof of Lemma 4.4)."""
    for seed in range(4):
        keys, res = _trace_case("uniform", 1 << 12, 24, 0.02, seed)
        for r in range(res.rounds + 1):
            L = res.trace_lrank[r].astype(np.int64)
            U = res.trace_urank[r].astype(np.int64)
            assert np.all(L[:-1] <= L[1:]) and np.all(U[:-1] <= U[1:])
            for i in range(len(L) - 1):
                same = L[i] == L[i + 1] and U[i] == U[i + 1]
                assert same or U[i] <= L[i + 1]
            if r > 0:
                assert np.all(res.trace_lrank[r] >= res.trace_lrank[r - 1])
                assert np.all(res.trace_urank[r] <= res.trace_urank[r - 1])


def test_round_with_q_one_resolves_everything():
    """Termination: once q = 1 every key of every unresolved interval is a
    probe, so every splitter resolves in that round."""
    hits = 0
    for seed in range(12):
        keys, res = _trace_case("uniform", 1 << 12, 16, 0.004, seed, oversample=5.0)
        for r in range(res.rounds):
            if 5.0 * 16 >= int(res.gamma[r]):
                assert int(res.unresolved[r + 1]) == 0
                assert r == res.rounds - 1
                hits += 1
    assert hits > 0


def test_sample_sizes_chernoff():
    """Z_j ~ Binomial(|gamma_{j-1}|, q_j); each round stays inside a 6-sigma
    band around its mean s*p (the Chernoff argument of Lemma 4.6)."""
    N, p = 1 << 14, 32
    for seed in range(10):
        res = oracle.hss(inputs.uniform(N, seed), p, 0.02, seed=seed, sort=False)
        for r in range(res.rounds):
            g = int(res.gamma[r])
            q = min(1.0, 5.0 * p / g)
            mean = q * g
            sd = math.sqrt(max(mean * (1 - q), 1e-9))
            assert abs(int(res.sample_size[r]) - mean) <= 6 * sd + 1


def test_gamma_shrinks_like_lemma_4_4():
    """E|gamma_j| <= 2N/s_j with the effective sampling ratio s_j = q_j N/p
    (Lemma 4.4), averaged over seeds (gamma here counts only unresolved
    intervals, a subset of the lemma's union)."""
    N, p, s = 1 << 14, 64, 5.0
    ratios = []
    for seed in range(30):
        res = oracle.hss(inputs.uniform(N, 100 + seed), p, 0.01, seed=seed, oversample=s, sort=False)
        for r in range(res.rounds - 1):
            g_prev, g_next = int(res.gamma[r]), int(res.gamma[r + 1])
            q = min(1.0, s * p / g_prev)
            if q >= 1.0:
                continue
            s_eff = q * N / p
            ratios.append(g_next / (2.0 * N / s_eff))
    assert len(ratios) > 20
    assert float(np.mean(ratios)) <= 1.05
    # the w.h.p. bound |gamma_j| <= 4N/s_j (Lemma 4.5) holds in every case
    assert max(ratios) <= 2.0


def test_rounds_logarithmic():
    """Rounds grow like log(log p / eps) (Theorem 4.8); at s = 5 the interval
    union shrinks ~s/2 per round, so rounds stay within a small window of
    ln(ln p/(s eps))/ln(s/2) + 1."""
    for p, eps in [(16, 0.05), (64, 0.02), (256, 0.02)]:
        N = p * 512
        rounds = [oracle.hss(inputs.uniform(N, seed), p, eps, seed=seed, sort=False).rounds for seed in range(6)]
        expect = math.log(math.log(p) / (5 * eps)) / math.log(2.5) + 1
        assert min(rounds) >= 1
        assert max(rounds) <= expect + 4, (p, eps, rounds, expect)


@pytest.mark.slow
def test_paper_round_count_p2048():
    """Sec. 7.2: at p = 2048 with 5p probes per round HSS converged in 6
    iterations.  Soft check of the same setting on synthetic keys."""
    with open(os.path.join(GOLDEN, "paper_round_counts.json")) as f:
        g = json.load(f)["single_stage_p2048"]
    p, s, eps = g["p"], g["probes_per_round_over_p"], g["eps_assumed"]
    N = p * 1024
    res = oracle.hss(inputs.uniform(N, 1), p, eps, seed=1, oversample=s, sort=False)
    assert res.status == 0
    assert abs(res.rounds - g["iterations"]) <= g["window"], res.rounds


def test_proposal_cuts_are_histogrammed():
    """Externally proposed non-member cuts enter L/U before round 1; the
    result still satisfies the contract and uses no more rounds."""
    N, p, eps = 1 << 14, 32, 0.02
    keys = inputs.uniform(N, 3)
    srt = np.sort(keys)
    prop = srt[[(i * N) // p for i in range(1, p)]]
    base = oracle.hss(keys, p, eps, seed=2)
    res = oracle.hss(keys, p, eps, seed=2, proposal=prop)
    assert res.status == 0
    _check_result(keys, p, eps, res)
    # exact proposals resolve every splitter before any sampling
    assert res.rounds == 0 and base.rounds >= 1


# ---------------------------------------------------------------------------
# The other sampling schedules: the k-round schedule of Theorem 4.7 and the
# equal-per-interval (HykSort) sampling the paper contrasts with in Sec. 4.2.2.
# ---------------------------------------------------------------------------
def _region(res, r, N, p):
    L = res.trace_lrank[r].astype(np.int64)
    U = res.trace_urank[r].astype(np.int64)
    flags = res.trace_resolved[r]
    resolved = (flags & 1) != 0
    lmem = (flags & 2) != 0
    ints = []
    done = set()
    for i in range(p - 1):
        if resolved[i]:
            continue
        lo, hi = int(L[i]) + int(lmem[i]), int(U[i])
        if (lo, hi) in done:
            continue
        done.add((lo, hi))
        ints.append((lo, hi))
    return ints


@pytest.mark.parametrize("schedule,k", [("theory", 2), ("theory", 3), ("equal", 0)])
def test_sampling_set_rederived_other_schedules(schedule, k):
    """Each round samples exactly the keys of the unresolved region whose
    Philox word is below the schedule's threshold: p s_j / N with
    s_j = (2 ln p / eps)^(j/k) (Theorem 4.7), or s p / nint spread equally
    over the nint distinct intervals (HykSort)."""
    N, p, eps, seed = 1 << 13, 16, 0.02, 5
    keys = inputs.uniform(N, seed)
    res = oracle.hss(keys, p, eps, seed=seed, trace=True, schedule=schedule, schedule_k=k)
    assert res.status == 0 and res.rounds >= 1
    b, idx = _sorted_pos_to_input_index(keys, p)
    _, rank_of = _global_order(keys, p)
    rank_sp = [rank_of[idx[s]] for s in range(p)]
    for r in range(res.rounds):
        ints = _region(res, r, N, p)
        assert sum(hi - lo for lo, hi in ints) == int(res.gamma[r])
        thr = {}
        for lo, hi in ints:
            if schedule == "theory":
                sj = math.pow(2.0 * math.log(p) / eps, min(r + 1, k) / k)
                q = (p * sj) / N
            else:
                q = (5.0 * p / len(ints)) / (hi - lo) if hi > lo else 1.0
            thr[(lo, hi)] = (True, 0) if q >= 1.0 else (False, int(math.floor(math.ldexp(q, 64))))
        want = set()
        for s in range(p):
            for spos in range(len(rank_sp[s])):
                rk = rank_sp[s][spos]
                for lo, hi in ints:
                    if lo <= rk < hi:
                        all_, T = thr[(lo, hi)]
                        if all_ or oracle.sample_draw(seed, s, spos, r + 1) < T:
                            want.add((s, spos))
        got = {(int(sg), int(sp)) for _, sg, sp in res.samples[r]}
        assert got == want


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_theory_one_round_is_lemma_4_1(seed):
    """k = 1: every key drawn with probability 2 p ln p / (eps N) puts a key
    in every target range w.h.p. (Lemma 4.1): one round."""
    N, p, eps = 1 << 16, 32, 0.05
    keys = inputs.uniform(N, seed)
    res = oracle.hss(keys, p, eps, seed=seed, schedule="theory", schedule_k=1)
    assert res.status == 0 and res.rounds == 1
    _check_result(keys, p, eps, res)


@pytest.mark.parametrize("k", [2, 3])
def test_theory_k_rounds_theorem_4_7(k):
    """With s_j = (2 ln p / eps)^(j/k) the splitters are found after k rounds
    w.h.p. (Lemma 4.3, Theorem 4.7), and round j draws about p s_j/N of the
    region (a 6-sigma Chernoff band)."""
    N, p, eps = 1 << 16, 64, 0.02
    for seed in (1, 2, 3):
        keys = inputs.gauss_mix(N, seed)
        res = oracle.hss(keys, p, eps, seed=seed, schedule="theory", schedule_k=k)
        assert res.status == 0 and res.rounds <= k
        _check_result(keys, p, eps, res)
        for j in range(res.rounds):
            q = min(1.0, p * math.pow(2.0 * math.log(p) / eps, (j + 1) / k) / N)
            mean = q * int(res.gamma[j])
            assert abs(int(res.sample_size[j]) - mean) <= 6.0 * math.sqrt(max(mean * (1 - q), 1e-9)) + 1


@pytest.mark.parametrize("gen", ["uniform", "gauss_mix"])
def test_equal_schedule_expected_probes_per_interval(gen):
    """Equal sampling per interval (the HykSort way, Sec. 4.2.2): interval u
    of length len_u draws Binomial(len_u, q_u) probes with
    q_u = min(1, (s p / nint) / len_u), so each interval expects s p / nint
    probes whatever its length.  Each interval's count lies in a 6-sigma
    Chernoff band, and the count pooled over rounds, intervals and seeds
    within 4 sigma of the pooled expectation (a dropped or misplaced nint
    shifts it by far more)."""
    N, p, eps, s = 1 << 13, 16, 0.02, 5.0
    g = {"uniform": inputs.uniform, "gauss_mix": inputs.gauss_mix}[gen]
    pooled_got = pooled_mean = pooled_var = 0.0
    for seed in range(1, 9):
        keys = g(N, seed)
        res = oracle.hss(keys, p, eps, seed=seed, trace=True, schedule="equal")
        assert res.status == 0
        _, idx = _sorted_pos_to_input_index(keys, p)
        _, rank_of = _global_order(keys, p)
        rank_sp = [rank_of[idx[q]] for q in range(p)]
        for r in range(res.rounds):
            ints = _region(res, r, N, p)
            cnt = {iv: 0 for iv in ints}
            for _, sg, sp in res.samples[r]:
                rk = rank_sp[int(sg)][int(sp)]
                hit = [iv for iv in ints if iv[0] <= rk < iv[1]]
                assert len(hit) == 1
                cnt[hit[0]] += 1
            for (lo, hi), c in cnt.items():
                ln = hi - lo
                q = min(1.0, (s * p / len(ints)) / ln) if ln > 0 else 1.0
                mean, var = q * ln, ln * q * (1.0 - q)
                assert abs(c - mean) <= 6.0 * math.sqrt(var) + 1.0
                if q < 1.0:
                    assert abs(mean - s * p / len(ints)) < 1e-6 * mean
                pooled_got += c
                pooled_mean += mean
                pooled_var += var
    assert abs(pooled_got - pooled_mean) <= 4.0 * math.sqrt(pooled_var) + 1.0


@pytest.mark.parametrize("gen,max_rounds", [("uniform", 1), ("uniform", 2), ("zipf", 1)])
def test_final_choice_is_closest_seen_cut(gen, max_rounds):
    """Sec. 4.2.2 step 5: each splitter is the seen cut ranked closest to t_i,
    over every probe of every round; with a round limit most splitters stay
    unresolved, so the choice (and its tie rule, equal distance -> L_i) is
    exercised.  Ranks of the probes are taken by brute force; the sentinels
    (rank 0 with no probe below, rank N with none above) are reported with
    seg -2 / -3."""
    N, p = 1 << 12, 16
    gens = {"uniform": inputs.uniform, "zipf": lambda n, s: inputs.zipf(n, s, distinct=200)}
    ties = 0
    for seed in range(60):
        keys = gens[gen](N, seed)
        res = oracle.hss(keys, p, 0.002, seed=seed, oversample=1.0, max_rounds=max_rounds, trace=True)
        assert res.rounds <= max_rounds
        order, rank_of = _global_order(keys, p)
        _, idx = _sorted_pos_to_input_index(keys, p)
        seen = np.array([rank_of[idx[int(sg)][int(sp)]] for r in range(res.rounds)
                         for _, sg, sp in res.samples[r]], dtype=np.int64)
        for i in range(p - 1):
            t = ((i + 1) * N) // p
            below, above = seen[seen <= t], seen[seen >= t]
            lo = int(below.max()) if below.size else 0
            hi = int(above.min()) if above.size else N
            want = lo if t - lo <= hi - t else hi
            ties += int(lo != hi and t - lo == hi - t)
            assert int(res.offsets[i + 1]) == want
            if want == 0 and not below.size:
                assert int(res.splitter_seg[i]) == -2
            elif want == N and not above.size:
                assert int(res.splitter_seg[i]) == -3
            else:
                e = idx[int(res.splitter_seg[i])][int(res.splitter_spos[i])]
                assert int(rank_of[e]) == want and keys[e] == res.splitter_key[i]
    assert ties >= 1  # the tie rule was reached


@pytest.mark.parametrize("gen", ["uniform", "zipf"])
def test_resolution_rule_against_brute_force(gen):
    """Sec. 4.2.2 step 3: after every round, splitter i counts as resolved
    exactly when the best probe seen so far below or above t_i (brute-force
    ranks) lies within tol = floor(N eps / 2p) of it, the bound inclusive;
    the per-round unresolved counts follow, and the rounds stop at the first
    round that leaves none.  Cases where only the equality |rank - t_i| = tol
    resolves a splitter occur and are checked."""
    N, p, eps = 1 << 13, 16, 0.02
    tol = (N * 2 // 100) // (2 * p)  # floor(N eps / 2p) in integers: eps = 2/100
    assert tol == 5
    gens = {"uniform": inputs.uniform, "zipf": lambda n, s: inputs.zipf(n, s, distinct=300)}
    decisive = 0
    for seed in range(20):
        keys = gens[gen](N, seed)
        res = oracle.hss(keys, p, eps, seed=seed, trace=True)
        assert res.tol == tol
        _, rank_of = _global_order(keys, p)
        _, idx = _sorted_pos_to_input_index(keys, p)
        seen = np.zeros(0, dtype=np.int64)
        for r in range(res.rounds + 1):
            if r:
                seen = np.concatenate([seen, np.array([rank_of[idx[int(sg)][int(sp)]]
                                                       for _, sg, sp in res.samples[r - 1]], dtype=np.int64)])
            open_ = 0
            for i in range(p - 1):
                t = ((i + 1) * N) // p
                below, above = seen[seen <= t], seen[seen >= t]
                dl = t - (int(below.max()) if below.size else 0)
                du = (int(above.min()) if above.size else N) - t
                ok = dl <= tol or du <= tol
                decisive += int(ok and min(dl, du) == tol)
                assert bool(res.trace_resolved[r, i] & 1) == ok
                assert bool(res.trace_resolved[r, i] & 2) == bool(below.size)  # L is an input key
                assert bool(res.trace_resolved[r, i] & 4) == bool(above.size)  # U is an input key
                open_ += int(not ok)
            assert int(res.unresolved[r]) == open_
            assert (open_ == 0) == (r == res.rounds)
    assert decisive >= 1
