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


def _bare_server(budget, reserve=0, available=0, slots=2):
    """A Server with only the fields admission reads (no device, no streams)."""
    from paper_1803_01237_gb300 import serve
    s = object.__new__(serve.Server)
    s.hbm_budget, s.hbm_reserve, s.pending_bytes, s.bytes_in_flight = budget, reserve, 0, 0
    s.slot_ws = [None] * slots
    s._available_bytes = lambda: available
    return s


class _Ws:
    def __init__(self, n):
        self.n = n

    def numel(self):
        return self.n


def test_admission_by_memory():
    """Admission rules of the server, on the host: no budget admits every
    request; a fixed budget counts the bytes of the requests in flight; the
    "free" budget compares what the request would allocate now (the slot's
    workspace growth plus its outputs) and what earlier admissions have yet to
    allocate with the device's available bytes less the reserve."""
    from paper_1803_01237_gb300 import serve
    import torch
    req = serve.Request(rid=0, arrival=0.0, keys=torch.zeros(1 << 20, dtype=torch.int64), p=256, eps=0.02, seed=1)
    nb = serve.Server.request_bytes(1 << 20, 256)
    need = nb + 4096  # outputs beyond the workspace
    assert _bare_server(None)._fits(0, req, need)
    s = _bare_server(need + 100)
    assert s._fits(0, req, need)
    s.bytes_in_flight = 101
    assert not s._fits(0, req, need)
    s = _bare_server("free", reserve=1000, available=need + 1000)
    assert s._growth(0, req, need) == need and s._fits(0, req, need)
    s.pending_bytes = 1
    assert not s._fits(0, req, need)
    s.slot_ws[1] = _Ws(nb)  # a slot whose cached workspace is large enough grows by the outputs only
    assert s._growth(1, req, need) == 4096 and s._fits(1, req, need)
    s.slot_ws[1] = _Ws(nb // 2)
    assert s._growth(1, req, need) == nb - nb // 2 + 4096
