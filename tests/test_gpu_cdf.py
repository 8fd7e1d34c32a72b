"""The CDF network kernels (hss_cdf_*) against the float64 oracle
(oracle/cdf_mlp.py), and what the trained network gains the rounds.

Tolerances: the kernels compute in float32 (inputs rounded to float32 from a
double-precision feature, sums of up to a few thousand terms), the oracle in
float64.  A float32 sum of n terms of relative rounding 2^-24 each differs
from the exact sum by at most about n 2^-24 of the sum of magnitudes; with
n <= 4096 that is below 2.5e-4 of max|g| per entry, and the tests allow
1e-3 relative plus 1e-4 of max|g| absolute.
"""
import numpy as np
import pytest

import oracle
import oracle.cdf_mlp as M
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


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _job(n, seed):
    keys = inputs.lognormal_job(n, seed)
    order = np.argsort(keys, kind="stable")
    ranks = np.empty(n, dtype=np.uint64)
    ranks[order] = np.arange(n, dtype=np.uint64)
    return keys, ranks


def _bounds(keys):
    return int(keys.min()), int(keys.max())


def _model(hss, keys, seed=3, feature="log"):
    lo, hi = _bounds(keys)
    m = hss.CDFModel().init(seed, feature, lo, hi)
    rlo = np.log2(1.0 + float(lo)) if feature == "log" else float(lo)
    rhi = np.log2(1.0 + float(hi)) if feature == "log" else float(hi)
    return m, rlo, rhi


def test_init_matches_oracle(hss):
    keys, _ = _job(1000, 1)
    for seed in (0, 3, 2**40 + 17):
        m, _, _ = _model(hss, keys, seed)
        assert np.allclose(m.theta.cpu().numpy(), M.init(seed), rtol=1e-6, atol=1e-7)
        assert m.step == 0


@pytest.mark.parametrize("n,feature", [(3000, "log"), (257, "linear"), (4096, "log")])
def test_gradient_matches_oracle(hss, n, feature):
    keys, ranks = _job(n, 5)
    N = n
    m, lo, hi = _model(hss, keys, 4, feature)
    theta = M.init(4) + 0.05 * np.random.default_rng(n).standard_normal(M.NPARAM)
    m.theta.copy_(torch.from_numpy(theta.astype(np.float32)))
    g, loss = m.grad(dev_u64(keys), dev_u64(ranks), N)
    x = M.feature(keys, M.LOG if feature == "log" else M.LINEAR, lo, hi)
    # the kernel's parameters are float32: give the oracle the same values
    th32 = m.theta.cpu().numpy().astype(np.float64)
    gref, Lref = M.grad(th32, x, ranks.astype(np.float64) / N)
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.abs(gref).max()
    assert np.allclose(gg, gref, rtol=1e-3, atol=1e-4 * scale)
    assert float(loss.item()) == pytest.approx(Lref, rel=1e-4)


def test_eval_matches_oracle(hss):
    keys, _ = _job(5000, 6)
    m, lo, hi = _model(hss, keys, 9)
    y = m.eval(dev_u64(keys)).cpu().numpy()
    yref, _ = M.forward(m.theta.cpu().numpy().astype(np.float64), M.feature(keys, M.LOG, lo, hi))
    assert np.allclose(y, yref, rtol=1e-4, atol=1e-5)


def test_adam_steps_match_oracle(hss):
    keys, ranks = _job(2000, 7)
    N = 2000
    m, lo, hi = _model(hss, keys, 11)
    th0 = m.theta.cpu().numpy().astype(np.float64)
    x = M.feature(keys, M.LOG, lo, hi)
    t = ranks.astype(np.float64) / N
    lr = 0.003
    m.train(dev_u64(keys), dev_u64(ranks), N, 1, lr)
    th1 = m.theta.cpu().numpy().astype(np.float64)
    g, _ = M.grad(th0, x, t)
    ref, _, _ = M.adam_step(th0, np.zeros(M.NPARAM), np.zeros(M.NPARAM), g, 1, lr)
    # first Adam step moves each parameter by about lr sign(g); where |g| is
    # within float32 noise of zero the sign itself is not determined
    clear = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.allclose(th1[clear], ref[clear], rtol=1e-5, atol=1e-6)
    assert np.all(np.abs(th1 - th0) <= lr * 1.0001 + 1e-7)
    assert m.step == 1


def test_training_fits_like_the_oracle(hss):
    keys, ranks = _job(4096, 8)
    N = 4096
    m, lo, hi = _model(hss, keys, 12)
    x = M.feature(keys, M.LOG, lo, hi)
    t = ranks.astype(np.float64) / N
    L0 = M.loss(m.theta.cpu().numpy().astype(np.float64), x, t)
    m.train(dev_u64(keys), dev_u64(ranks), N, 300, 0.01)
    torch.cuda.synchronize()
    Lgpu = M.loss(m.theta.cpu().numpy().astype(np.float64), x, t)
    _, _, _, Lref = M.train(M.init(12), x, t, 300, 0.01)
    assert Lgpu < 0.01 * L0
    assert Lgpu < 3.0 * Lref + 1e-5
    assert m.step == 300


def test_proposal_inverts_the_network(hss):
    """Each proposed key x_i satisfies y(x_i) >= i/p and y just below it < i/p
    (bisection), checked with the oracle's forward on the trained network."""
    keys, ranks = _job(4096, 13)
    m, lo, hi = _model(hss, keys, 14)
    m.train(dev_u64(keys), dev_u64(ranks), 4096, 200, 0.01)
    p = 64
    prop = m.propose(p).cpu().numpy().view(np.uint64)
    assert prop.shape == (p - 1,)
    th = m.theta.cpu().numpy().astype(np.float64)
    x = M.feature(prop, M.LOG, lo, hi)
    y, _ = M.forward(th, x)
    tau = np.arange(1, p) / p
    assert np.all(y >= tau - 1e-4)
    assert np.all(np.diff(prop.astype(np.float64)) >= 0)  # a trained CDF is monotone here


def test_identity_network_proposes_uniform_quantiles(hss):
    lo_key, hi_key = 1000, 1000 + (1 << 40)
    m = hss.CDFModel().init(1, "linear", lo_key, hi_key)
    w1 = np.zeros(M.H); w1[0] = 1.0
    W2 = np.zeros((M.H, M.H)); W2[0, 0] = 1.0
    w3 = np.zeros(M.H); w3[0] = 1.0
    th = M.pack(w1, np.zeros(M.H), W2, np.zeros(M.H), w3, 0.0)
    m.theta.copy_(torch.from_numpy(th.astype(np.float32)))
    p = 16
    prop = m.propose(p).cpu().numpy().view(np.uint64).astype(np.float64)
    want = lo_key + np.arange(1, p) / p * (hi_key - lo_key)
    assert np.all(np.abs(prop - want) <= 2.0 ** 40 * 2.0 ** -22)


def test_proposal_with_several_cuts_per_splitter(hss):
    """per_splitter cuts at targets i/p + delta (2k/(per-1) - 1): the oracle's
    network output at each proposed key reaches its target, and the cuts of
    one splitter are ordered."""
    keys, ranks = _job(4096, 15)
    m, lo, hi = _model(hss, keys, 16)
    m.train(dev_u64(keys), dev_u64(ranks), 4096, 200, 0.01)
    p, per, delta = 32, 5, 0.004
    prop = m.propose(p, per, delta).cpu().numpy().view(np.uint64)
    assert prop.shape == ((p - 1) * per,)
    th = m.theta.cpu().numpy().astype(np.float64)
    y, _ = M.forward(th, M.feature(prop, M.LOG, lo, hi))
    tau = M.targets(p, per, delta)
    assert np.all(y >= tau - 1e-4)
    assert np.all(np.diff(prop.reshape(p - 1, per).astype(np.float64), axis=1) >= 0)


def test_trained_network_saves_rounds(hss):
    """Train on the splitters (exact ranks of sampled keys) of earlier
    lognormal jobs, propose 16 cuts per splitter around the predicted
    quantiles for the next job of the same stream: the histogram of those
    cuts brackets every target rank from both sides before any sampling, so
    fewer rounds are needed, and the result is still the oracle's for the
    same proposed cuts."""
    N, p, eps = 1 << 20, 256, 0.02
    m = None
    tk_all, tr_all = [], []
    rounds_plain, rounds_prop = [], []
    loss = None
    for j in range(5):
        keys = inputs.lognormal_job(N, 100 + j)
        dk = dev_u64(keys)
        plain, _ = hss.partition(dk, p, eps, 1)
        if m is not None:
            delta = max(3.0 * float(loss) ** 0.5, 0.25 / p)
            prop = m.propose(p, 16, delta)
            res, _ = hss.partition_with_proposal(dk, p, eps, 1, prop)
            rounds_plain.append(plain.rounds)
            rounds_prop.append(res.rounds)
            if j == 4:
                ref = oracle.hss(keys, p, eps, 1, sort=False, proposal=prop.cpu().numpy().view(np.uint64))
                assert res.rounds == ref.rounds and res.sample_size == [int(x) for x in ref.sample_size]
                assert np.array_equal(res.offsets.cpu().numpy().astype(np.uint64), ref.offsets)
        else:
            m = hss.CDFModel().init(5, "log", int(keys.min()), int(keys.max()))
        tk, tr = hss.training_pairs(plain)
        tk_all.append(tk)
        tr_all.append(tr)
        loss = m.train(torch.cat(tk_all), torch.cat(tr_all), N, 300, 0.01).item()
    print("rounds plain", rounds_plain, "with proposal", rounds_prop, "last training loss", loss)
    assert sum(rounds_prop) < sum(rounds_plain)
    assert max(rounds_prop) < max(rounds_plain)


def test_gpu_bisection_returns_the_smallest_x(hss):
    """A network flat at 1/2 on [1/2, 3/4]: every x there has y(x) >= 1/2, and
    the proposal for tau = 1/2 is the smallest such x (1/2), as in the
    oracle's bisection; tau = 1/4 and 3/4 land at 1/4 and 1."""
    lo_key, hi_key = 0, 1 << 40
    m = hss.CDFModel().init(1, "linear", lo_key, hi_key)
    w1 = np.zeros(M.H); b1 = np.zeros(M.H)
    w1[0], w1[1], b1[1], w1[2], b1[2] = 1.0, 1.0, -0.5, 1.0, -0.75
    W2 = np.zeros((M.H, M.H)); W2[0, 0], W2[0, 1], W2[1, 2] = 1.0, -1.0, 1.0
    w3 = np.zeros(M.H); w3[0], w3[1] = 1.0, 1.0
    th = M.pack(w1, b1, W2, np.zeros(M.H), w3, 0.0)
    m.theta.copy_(torch.from_numpy(th.astype(np.float32)))
    prop = m.propose(4).cpu().numpy().view(np.uint64).astype(np.float64)
    want = np.array([0.25, 0.5, 1.0]) * float(hi_key)
    assert np.all(np.abs(prop - want) <= float(hi_key) * 2.0 ** -22)
    ref = M.propose(th, 4, M.LINEAR, float(lo_key), float(hi_key)).astype(np.float64)
    assert np.all(np.abs(prop - ref) <= float(hi_key) * 2.0 ** -22)


# ---------------------------------------------------------------------------
# The bfloat16 weight variant: every evaluation uses the parameters rounded to
# bfloat16; the oracle is the same float64 network on M.round_bf16(theta).
# ---------------------------------------------------------------------------
def test_bf16_eval_and_gradient_match_the_oracle(hss):
    keys, ranks = _job(3000, 21)
    N = 3000
    m, lo, hi = _model(hss, keys, 22)
    theta = M.init(22) + 0.05 * np.random.default_rng(5).standard_normal(M.NPARAM)
    m.theta.copy_(torch.from_numpy(theta.astype(np.float32)))
    m.set_weights("bf16")
    x = M.feature(keys, M.LOG, lo, hi)
    th32 = m.theta.cpu().numpy().astype(np.float64)
    thb = M.round_bf16(th32)
    assert not np.array_equal(thb, th32)  # the rounding changes the network
    y = m.eval(dev_u64(keys)).cpu().numpy()
    yb, _ = M.forward(thb, x)
    assert np.allclose(y, yb, rtol=1e-4, atol=1e-5)
    y32, _ = M.forward(th32, x)
    assert np.abs(yb - y32).max() > 1e-4  # and the kernel followed it, not the float32 weights
    g, loss = m.grad(dev_u64(keys), dev_u64(ranks), N)
    gref, Lref = M.grad(thb, x, ranks.astype(np.float64) / N)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.allclose(gg, gref, rtol=1e-3, atol=1e-4 * np.abs(gref).max())
    assert float(loss.item()) == pytest.approx(Lref, rel=1e-4)
    m.set_weights("fp32")
    y2 = m.eval(dev_u64(keys)).cpu().numpy()
    assert np.allclose(y2, y32, rtol=1e-4, atol=1e-5)


def test_bf16_training_fits_and_proposes(hss):
    """Training through the bfloat16 weights (float32 master copy) fits the
    CDF about as well as float32, and its proposals invert the rounded
    network."""
    keys, ranks = _job(4096, 23)
    N = 4096
    m, lo, hi = _model(hss, keys, 24)
    m.set_weights("bf16")
    x = M.feature(keys, M.LOG, lo, hi)
    t = ranks.astype(np.float64) / N
    L0 = M.loss(M.round_bf16(m.theta.cpu().numpy()), x, t)
    m.train(dev_u64(keys), dev_u64(ranks), N, 300, 0.01)
    torch.cuda.synchronize()
    thb = M.round_bf16(m.theta.cpu().numpy())
    Lb = M.loss(thb, x, t)
    _, _, _, Lref = M.train(M.init(24), x, t, 300, 0.01)
    assert Lb < 0.01 * L0
    assert Lb < 3.0 * Lref + 1e-5
    p = 64
    prop = m.propose(p).cpu().numpy().view(np.uint64)
    y, _ = M.forward(thb, M.feature(prop, M.LOG, lo, hi))
    assert np.all(y >= np.arange(1, p) / p - 1e-4)
