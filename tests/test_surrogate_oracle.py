"""Pins of the surrogate oracle (oracle/mlp.py) against things other than itself."""
import numpy as np
import scipy.stats

from oracle import mlp as M
from paper_2502_11129_b300 import population as P


def small_params(rng, hidden=6, in_dim=5):
    return dict(W1=rng.normal(size=(hidden, in_dim)), b1=rng.normal(size=hidden) * 0.1,
                W2=rng.normal(size=(hidden, hidden)), b2=rng.normal(size=hidden) * 0.1,
                W3=rng.normal(size=(1, hidden)), b3=rng.normal(size=1))


def test_gradients_match_central_finite_differences():
    """Every gradient entry against (L(p + h e) - L(p - h e)) / 2h.  Weights are
    BF16-representable so the rounding inside forward is the identity."""
    rng = np.random.default_rng(0)
    p = {k: M.bf16_round(v) for k, v in small_params(rng).items()}
    X = M.bf16_round(rng.normal(size=(9, 5)))
    t = rng.normal(size=9)
    g, _ = M.backward(p, X, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for j in range(flat.size):
            if k.startswith("W"):
                continue  # perturbed weights leave the BF16 grid; checked below
            pp = {q: v.copy() for q, v in p.items()}
            pm = {q: v.copy() for q, v in p.items()}
            pp[k].reshape(-1)[j] += h
            pm[k].reshape(-1)[j] -= h
            fd = (M.loss(pp, X, t) - M.loss(pm, X, t)) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[j]) < 1e-6 * max(1.0, abs(fd))
    # weights: finite differences with the BF16 rounding switched off
    orig = M.bf16_round
    try:
        M.bf16_round = lambda a: np.asarray(a, dtype=np.float64)
        g2, _ = M.backward(p, X, t)
        for k in ("W1", "W2", "W3"):
            flat = p[k].reshape(-1)
            for j in range(flat.size):
                pp = {q: v.copy() for q, v in p.items()}
                pm = {q: v.copy() for q, v in p.items()}
                pp[k].reshape(-1)[j] += h
                pm[k].reshape(-1)[j] -= h
                fd = (M.loss(pp, X, t) - M.loss(pm, X, t)) / (2 * h)
                assert abs(fd - g2[k].reshape(-1)[j]) < 1e-6 * max(1.0, abs(fd))
    finally:
        M.bf16_round = orig


def test_forward_hand_worked():
    """2-2-2-1 network worked by hand: x = (1, -2);
    z1 = (1*1 + 0.5*-2 + 0.25, -1*1 + 1*-2 + 0) = (0.25, -3) -> h1 = (0.25, 0)
    z2 = (2*0.25 + 1*0 - 0.5, 1*0.25 + 4*0 + 1) = (0, 1.25) -> h2 = (0, 1.25)
    y = 3*0 - 2*1.25 + 0.5 = -2."""
    p = dict(W1=np.array([[1.0, 0.5], [-1.0, 1.0]]), b1=np.array([0.25, 0.0]),
             W2=np.array([[2.0, 1.0], [1.0, 4.0]]), b2=np.array([-0.5, 1.0]),
             W3=np.array([[3.0, -2.0]]), b3=np.array([0.5]))
    y, c = M.forward(p, np.array([[1.0, -2.0]]))
    assert y[0] == -2.0
    assert np.array_equal(c["h1"][0], [0.25, 0.0])


def test_bf16_rounding_is_nearest_even():
    assert M.bf16_round(np.array([1.0]))[0] == 1.0
    # 1 + 2^-8 is exactly halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert M.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert M.bf16_round(np.array([-3.0]))[0] == -3.0


def test_adam_first_step_is_lr_times_sign():
    """Kingma & Ba: at t = 1 the bias-corrected step is lr * g / (|g| + eps)."""
    p = dict(a=np.array([1.0, -2.0, 0.5]))
    g = dict(a=np.array([0.3, -0.01, 2.0]))
    m = dict(a=np.zeros(3))
    v = dict(a=np.zeros(3))
    p2, m2, v2 = M.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p2["a"], p["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), atol=1e-15)
    assert np.allclose(m2["a"], 0.1 * g["a"]) and np.allclose(v2["a"], 0.001 * g["a"] ** 2)


def test_adam_constant_gradient_steps_lr_at_every_t():
    """Kingma & Ba 2015: with m = v = 0 at the start and a constant gradient g,
    m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the bias-corrected moments
    are exactly g and g^2 and every step is lr * g / (|g| + eps); a wrong
    exponent in either correction breaks this at t = 2 and t = 3."""
    g = dict(a=np.array([0.3, -0.01, 2.0, -7.5]))
    p = dict(a=np.array([1.0, -2.0, 0.5, 0.0]))
    m = dict(a=np.zeros(4))
    v = dict(a=np.zeros(4))
    lr = 0.01
    step = lr * g["a"] / (np.abs(g["a"]) + 1e-8)
    for t in (1, 2, 3):
        p2, m, v = M.adam_step(p, g, m, v, t, lr=lr)
        assert np.allclose(p2["a"] - p["a"], -step, rtol=1e-12, atol=1e-15), t
        assert np.allclose(m["a"], (1 - 0.9 ** t) * g["a"], rtol=1e-12), t
        assert np.allclose(v["a"], (1 - 0.999 ** t) * g["a"] ** 2, rtol=1e-12), t
        p = p2


def test_adam_corrected_moments_are_normalised_weighted_means():
    """The bias-corrected first moment after t steps is the mean of the
    gradients seen so far weighted by b1^(t - i), normalised to sum 1 (the
    weights (1 - b1) b1^(t - i) sum to 1 - b1^t); the second moment likewise
    with b2 and g^2.  Checked through the parameter path of steps 1, 2, 3 with
    changing gradients."""
    b1, b2, eps, lr = 0.9, 0.999, 1e-8, 0.05
    gs = [np.array([1.0, -3.0]), np.array([2.0, 0.5]), np.array([4.0, -1.0])]
    p = dict(a=np.array([0.2, 0.7]))
    m = dict(a=np.zeros(2))
    v = dict(a=np.zeros(2))
    x = p["a"].copy()
    for t in (1, 2, 3):
        p, m, v = M.adam_step(p, dict(a=gs[t - 1]), m, v, t, lr=lr)
        w1 = np.array([b1 ** (t - i) for i in range(1, t + 1)])
        w2 = np.array([b2 ** (t - i) for i in range(1, t + 1)])
        G = np.array(gs[:t])
        mh = (w1[:, None] * G).sum(axis=0) / w1.sum()
        vh = (w2[:, None] * G ** 2).sum(axis=0) / w2.sum()
        x = x - lr * mh / (np.sqrt(vh) + eps)
        assert np.allclose(p["a"], x, rtol=1e-12, atol=1e-15), t


def test_encoding_of_a_hand_built_quadruped():
    pop = P.quadrupeds(1)
    x = M.encode_population(pop)[0]
    # bricks 1..4 are hips on core faces 0..3 (rotations 1, 1, 0, 0), 5..8 knees
    # on face 0 of hips 1..4 (rotation 1); slots 9..19 empty
    for i in range(8):
        b = i + 1
        assert x[5 * i] == 1.0
        assert x[5 * i + 1] == (0 if b <= 4 else b - 4) / 20.0
        assert x[5 * i + 2] == (b - 1 if b <= 4 else 0) / 5.0
        assert x[5 * i + 3] == ([1, 1, 0, 0][b - 1] if b <= 4 else 1) / 3.0
        assert x[5 * i + 4] == pop.w_int[0, b]
    assert np.all(x[40:100] == 0.0)
    # coupling weights: bricks 2..8 in slots 100..106; hips couple to the core -> 0
    assert np.all(x[100:103] == 0.0)
    assert np.allclose(x[103:107], pop.w_cpl[0, 5:9])
    assert np.all(x[107:] == 0.0)


def test_topk_against_full_sort_with_ties():
    rng = np.random.default_rng(1)
    s = rng.integers(0, 50, size=1000).astype(float)
    k = 100
    idx = M.topk(s, k)
    ref = sorted(range(len(s)), key=lambda i: (-s[i], i))[:k]
    assert list(idx) == ref


def test_spearman_against_library_and_monotone_invariance():
    rng = np.random.default_rng(2)
    a = rng.normal(size=300)
    b = a + rng.normal(size=300)
    b[::7] = b[3]  # ties
    assert abs(M.spearman(a, b) - scipy.stats.spearmanr(a, b).statistic) < 1e-12
    assert abs(M.spearman(a, np.exp(3 * a)) - 1.0) < 1e-12
    assert abs(M.spearman(a, -a ** 3) + 1.0) < 1e-12
