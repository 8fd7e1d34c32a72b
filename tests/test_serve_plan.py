"""Host logic of the server's proposal plan (no GPU): the expected-rounds
model against the oracle's actual round counts, and the choice of cuts per
splitter."""
import math

import numpy as np
import pytest

import oracle
from paper_1803_01237_gb300 import inputs, serve


def test_rounds_from_window():
    # an interval already inside the 2 tol window needs no round
    assert serve.rounds_from(0.02 / 64, 64, 0.02) == 0
    assert serve.rounds_from(0.019 / 64, 64, 0.02) == 0
    assert serve.rounds_from(2 * 0.02 / 64, 64, 0.02) == 1
    # each round shrinks by s: one factor of s beyond the window, plus margin
    assert serve.rounds_from(5 * 0.02 / 64, 64, 0.02) == 2
    assert serve.rounds_from(5.01 * 0.02 / 64, 64, 0.02) == 3


@pytest.mark.parametrize("p,eps", [(16, 0.02), (64, 0.02), (256, 0.02), (256, 0.2), (64, 0.005)])
def test_plain_rounds_model_matches_oracle(p, eps):
    """The plain-HSS prediction is within one round of what the method takes."""
    N = 1 << 16
    plain = serve.plain_rounds(p, eps)
    got = [oracle.hss(inputs.uniform(N, 10 + t), p, eps, t, sort=False).rounds for t in range(3)]
    assert all(abs(g - plain) <= 1 for g in got), (plain, got)


def _band_cuts(sorted_keys, p, per, delta, seed):
    """per non-member cuts per splitter at the quantiles i/p + e_i + delta
    (2k/(per-1) - 1), as a model whose error e_i at splitter i lies within
    +-delta/2 would propose (e_i uniform)."""
    N = sorted_keys.shape[0]
    err = np.random.default_rng(seed).uniform(-delta / 2, delta / 2, p)
    out = []
    for i in range(1, p):
        for k in range(per):
            tau = min(max(i / p + err[i] + delta * (2.0 * k / (per - 1) - 1.0), 0.0), 1.0)
            out.append(sorted_keys[min(N - 1, int(tau * N))])
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("p,delta", [(16, 4e-3), (64, 2e-3), (64, 0.25 / 64), (256, 1e-3)])
def test_planned_proposal_rounds_match_oracle(p, delta):
    """With the planned number of cuts per splitter, the oracle's sampling
    rounds after the proposal stay within one of the plan's prediction, and
    below the plain rounds."""
    N, eps = 1 << 16, 0.02
    per, r, plain = serve.plan_proposal(p, eps, delta, 16)
    assert per >= 2 and r < plain
    for t in range(3):
        keys = inputs.uniform(N, 40 + t)
        cuts = _band_cuts(np.sort(keys), p, per, delta, t)
        res = oracle.hss(keys, p, eps, t, sort=False, proposal=cuts)
        assert res.status == 0
        assert abs(res.rounds - (r - 1)) <= 1, (res.rounds, r)
        assert res.rounds < plain


def test_plan_choice():
    eps = 0.02
    # too coarse a model: plain HSS
    assert serve.plan_proposal(1024, eps, 0.01, 16)[0] == 0
    assert serve.plan_proposal(4096, eps, 1e-3, 16)[0] == 0
    for p in (32, 128, 512, 2048):
        for delta in (0.25 / p, 1.0 / p, 1e-3):
            per, r, plain = serve.plan_proposal(p, eps, delta, 16)
            if per == 0:
                continue
            assert r < plain
            assert (p - 1) * per <= 5 * p * (1 + plain - r)
            # the smallest per that reaches r
            for q in range(2, per):
                assert 1 + serve.rounds_from(2 * delta / (q - 1), p, eps) > r
            # a tighter model never needs more cuts or more rounds
            per2, r2, _ = serve.plan_proposal(p, eps, delta / 2, 16)
            assert per2 != 0 and r2 <= r
            assert r2 < r or per2 <= per


def test_delta_scales_with_job_size():
    d = serve.Server._dkw
    assert d(1 << 16) == pytest.approx(math.sqrt(math.log(200.0) / 2.0 ** 17))
    assert d(1 << 20) == pytest.approx(d(1 << 16) / 4)
