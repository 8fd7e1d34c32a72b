"""Pins of the CDF-network oracle (oracle/cdf_mlp.py) to what fixes it from
outside: finite differences of the loss, closed forms, the Adam paper's
first step, exact feature values and a network that is the identity."""
import numpy as np
import pytest

import oracle
import oracle.cdf_mlp as M


def _data(n, seed):
    g = np.random.default_rng(seed)
    x = g.random(n)
    t = np.clip(x ** 2 + 0.05 * g.standard_normal(n), 0.0, 1.0)
    return x, t


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    """The hand-written backward pass equals the numerical derivative of the
    loss (central differences in float64) for every one of the 1153
    parameters."""
    theta = M.init(seed)
    theta = theta + 0.01 * np.random.default_rng(seed).standard_normal(M.NPARAM)
    x, t = _data(64, seed)
    g, _ = M.grad(theta, x, t)
    h = 1e-6
    num = np.empty(M.NPARAM)
    for k in range(M.NPARAM):
        e = np.zeros(M.NPARAM)
        e[k] = h
        num[k] = (M.loss(theta + e, x, t) - M.loss(theta - e, x, t)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_closed_form_with_silent_hidden_layer():
    """W2 = 0: hidden-2 is relu(b2) for every input, y = w3.relu(b2) + b3 is
    constant, and only w3, b2 (through relu'), b3 get gradient."""
    w1 = np.linspace(-1, 1, M.H)
    b1 = np.full(M.H, 0.3)
    W2 = np.zeros((M.H, M.H))
    b2 = np.linspace(-0.5, 0.5, M.H)
    w3 = np.linspace(0.1, 0.4, M.H)
    theta = M.pack(w1, b1, W2, b2, w3, 0.25)
    x, t = _data(50, 7)
    g, L = M.grad(theta, x, t)
    y = float(w3 @ np.maximum(b2, 0.0) + 0.25)
    assert L == pytest.approx(np.mean((y - t) ** 2), rel=1e-12)
    dy = 2.0 * np.mean(y - t)
    gw1, gb1, gW2, gb2, gw3, gb3 = M.unpack(g)
    assert gb3 == pytest.approx(dy, rel=1e-12)
    assert np.allclose(gw3, dy * np.maximum(b2, 0.0), rtol=1e-12)
    assert np.allclose(gb2, dy * w3 * (b2 > 0), rtol=1e-12)
    assert np.allclose(gw1, 0.0) and np.allclose(gb1, 0.0)
    h1 = np.maximum(np.outer(x, w1) + b1, 0.0)
    d = 2.0 * (y - t) / x.shape[0]
    assert np.allclose(gW2, np.outer(w3 * (b2 > 0), d @ h1), rtol=1e-10)


def test_adam_first_step_is_signed_learning_rate():
    """From m = v = 0 the bias-corrected first step is -lr g / (|g| + eps)
    (Kingma and Ba, Sec. 2): about -lr sign(g)."""
    g = np.linspace(-3, 3, M.NPARAM)
    theta = np.zeros(M.NPARAM)
    th, m, v = M.adam_step(theta, np.zeros(M.NPARAM), np.zeros(M.NPARAM), g, 1, 0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + M.ADAM_EPS), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_feature_map_values():
    lo, hi = 10.0, 50.0
    keys = np.array([(1 << 10) - 1, (1 << 30) - 1, (1 << 50) - 1, 0, (1 << 62)], dtype=np.uint64)
    f = M.feature(keys, M.LOG, lo, hi)
    assert np.allclose(f[:3], [0.0, 0.5, 1.0], atol=1e-12)
    assert f[3] == 0.0 and f[4] == 1.0          # clipped
    f = M.feature(np.array([100, 150, 200], dtype=np.uint64), M.LINEAR, 100.0, 200.0)
    assert np.allclose(f, [0.0, 0.5, 1.0])
    # int64 keys use the order-preserving bits: -2^63 -> 0, 0 -> 2^63
    fi = M.feature(np.array([-(1 << 63), 0], dtype=np.int64), M.LINEAR, 0.0, 2.0 ** 64, key_type="i64")
    assert np.allclose(fi, [0.0, 0.5])


def _identity_net():
    """y = relu(relu(x)) = x on [0, 1]."""
    w1 = np.zeros(M.H); w1[0] = 1.0
    W2 = np.zeros((M.H, M.H)); W2[0, 0] = 1.0
    w3 = np.zeros(M.H); w3[0] = 1.0
    return M.pack(w1, np.zeros(M.H), W2, np.zeros(M.H), w3, 0.0)


def test_proposal_of_identity_network_is_uniform_quantiles():
    theta = _identity_net()
    lo, hi = 1000.0, 1000.0 + 2.0 ** 40
    p = 16
    keys = M.propose(theta, p, M.LINEAR, lo, hi)
    want = np.array([int(lo + (i / p) * (hi - lo)) for i in range(1, p)], dtype=np.uint64)
    assert np.all(np.abs(keys.astype(np.float64) - want.astype(np.float64)) <= 2.0 ** 40 * 2.0 ** -38)
    # LOG map: quantile i/p -> 2^(lo + (i/p)(hi-lo)) - 1
    kl = M.propose(theta, 4, M.LOG, 20.0, 60.0)
    assert np.allclose(np.log2(kl.astype(np.float64) + 1.0), [30.0, 40.0, 50.0], atol=1e-9)


def test_training_reduces_loss_and_fits_a_cdf():
    """Full-batch Adam on the empirical CDF of lognormal keys on the LOG map
    brings the mean squared error well below that of the initial network."""
    from paper_1803_01237_gb300 import inputs
    keys = np.sort(inputs.lognormal_job(4096, 5))
    ranks = np.arange(keys.shape[0], dtype=np.float64)
    lo, hi = np.log2(1.0 + float(keys[0])), np.log2(1.0 + float(keys[-1]))
    x = M.feature(keys, M.LOG, lo, hi)
    t = ranks / keys.shape[0]
    theta = M.init(3)
    L0 = M.loss(theta, x, t)
    theta, m, v, L = M.train(theta, x, t, 300, 0.01)
    assert L < 0.01 * L0 and L < 1e-3


def test_init_uses_the_philox_words():
    th = M.init(77)
    x = oracle.philox4x32_10((0, 0, 0, M.INIT_TAG), (77, 0))
    u0 = float(int(x[0]) >> 8) * 2.0 ** -24
    assert th[0] == pytest.approx((1.0 + u0) * 4.0, rel=1e-15)
    assert th[M.H] == pytest.approx(-th[0] * 0.5 / M.H, rel=1e-15)
    assert th[-1] == 0.5


def test_targets_several_cuts_per_splitter_hand_case():
    """per > 1: the cuts of splitter i sit at i/p + delta (2k/(per-1) - 1),
    k = 0..per-1, splitter-major, clipped to [0, 1] (worked by hand)."""
    got = M.targets(4, 3, 0.05)
    want = [0.20, 0.25, 0.30, 0.45, 0.50, 0.55, 0.70, 0.75, 0.80]
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    assert np.array_equal(M.targets(2, 2, 0.6), [0.0, 1.0])  # both ends clipped
    assert np.array_equal(M.targets(3, 1, 0.3), [1.0 / 3.0, 2.0 / 3.0])  # delta unused for one cut


def test_identity_network_proposes_targets_for_several_cuts():
    """The identity network y(x) = x proposes, for every target tau, the key
    at feature tau: lo + tau (hi - lo) on the linear map."""
    theta = _identity_net()
    lo, hi = 1000.0, 1000.0 + 2.0 ** 40
    keys = M.propose(theta, 4, M.LINEAR, lo, hi, per=3, delta=0.05)
    want = np.array([lo + t * (hi - lo) for t in [0.20, 0.25, 0.30, 0.45, 0.50, 0.55, 0.70, 0.75, 0.80]])
    assert np.all(np.abs(keys.astype(np.float64) - want) <= 2.0 ** 40 * 2.0 ** -38)


def _plateau_net():
    """y(x) = min(x, 1/2) + relu(x - 3/4) on [0, 1]: flat at 1/2 on [1/2, 3/4]."""
    w1 = np.zeros(M.H); b1 = np.zeros(M.H)
    w1[0], w1[1], b1[1], w1[2], b1[2] = 1.0, 1.0, -0.5, 1.0, -0.75   # relu(x), relu(x-1/2), relu(x-3/4)
    W2 = np.zeros((M.H, M.H))
    W2[0, 0], W2[0, 1] = 1.0, -1.0   # relu(relu(x) - relu(x-1/2)) = min(x, 1/2)
    W2[1, 2] = 1.0                   # relu(relu(x-3/4))
    w3 = np.zeros(M.H); w3[0], w3[1] = 1.0, 1.0
    return M.pack(w1, b1, W2, np.zeros(M.H), w3, 0.0)


def test_bisection_returns_the_smallest_x():
    """Where the network is flat at the target, every x of the plateau has
    y(x) >= tau; the proposal is the smallest one (x = 1/2 for tau = 1/2, not
    a point inside [1/2, 3/4]), and y just below it stays under tau."""
    theta = _plateau_net()
    xs = np.array([0.0, 0.25, 0.5, 0.6, 0.75, 0.9, 1.0])
    y, _ = M.forward(theta, xs)
    assert np.allclose(y, [0.0, 0.25, 0.5, 0.5, 0.5, 0.65, 0.75])
    lo, hi = 0.0, 2.0 ** 40
    keys = M.propose(theta, 2, M.LINEAR, lo, hi)   # tau = 1/2
    assert abs(float(keys[0]) - 0.5 * hi) <= 1.0
    x = M.feature(keys, M.LINEAR, lo, hi)
    assert M.forward(theta, x - 2.0 ** -30)[0][0] < 0.5 <= M.forward(theta, x + 2.0 ** -30)[0][0]


def test_bf16_rounding_hand_cases_and_library():
    """bfloat16 keeps the top 16 bits of a float32, rounded to nearest with
    ties to even: hand-worked values, then against torch's conversion."""
    one = 1.0
    cases = [
        (one, one),
        (one + 2.0 ** -8, one),                    # halfway, 1.0 has an even last bit: down
        (one + 3 * 2.0 ** -8, one + 2.0 ** -6),    # halfway, 1 + 2^-7 is odd: up
        (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7),  # above halfway: up
        (-(one + 2.0 ** -9), -one),                # below halfway: down (magnitude)
        (0.1, 0.10009765625),
        (3.0e38, 2.0 ** 127 * 226 / 128),          # 3e38 = 2^127 x 1.7633: 225.7/128 -> 226/128
    ]
    for x, want in cases:
        assert M.round_bf16(np.array([x]))[0] == want, x
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(3)
    x = np.concatenate([g.normal(size=4000), g.normal(size=4000) * 1e-30, g.uniform(-1e30, 1e30, 4000)])
    x32 = x.astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(M.round_bf16(x32), want)
