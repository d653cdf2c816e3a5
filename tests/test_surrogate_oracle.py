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
    """Zero-pose geometry written out by hand: hips (bodies 1..4) on the
    core's +x, -x, +y, -y faces, box centres 50 + 30 mm out, hinge axes
    vertical; knees (5..8) on each hip's outer face, centres 50 + 60 + 30 mm
    out, hinge axes horizontal across the leg (y for the x legs, x for the y
    legs).  All centres lie at z = 0, so the (z, x, y) order is by x, then y."""
    pop = P.quadrupeds(1)
    x = M.encode_population(pop)[0]
    # (body, centre in mm, axis code)
    expect = [(6, (-140, 0, 0), 2), (2, (-80, 0, 0), 3), (8, (0, -140, 0), 1), (4, (0, -80, 0), 3),
              (3, (0, 80, 0), 3), (7, (0, 140, 0), 1), (1, (80, 0, 0), 3), (5, (140, 0, 0), 2)]
    for i, (b, c, code) in enumerate(expect):
        f = x[6 * i:6 * i + 6]
        assert np.array_equal(f[:3], np.array(c) / 256.0), (i, b, f)
        assert f[3] == code / 3.0, (i, b)
        assert f[4] == pop.w_int[0, b]
        # knees couple to their hip; hips hang off the core (no coupling)
        assert f[5] == (pop.w_cpl[0, b] if b >= 5 else 0.0)
    assert np.all(x[48:] == 0.0)


def test_encoding_sorts_and_ignores_build_order():
    """The same robot built in another order (bricks renumbered, parents
    before children) encodes identically; a brick moved by one lattice step
    moves its slot's centre by 1/256 and nothing else."""
    pop = P.grammar(1, seed=11)
    nb = int(pop.nb[0])
    R9 = pop.R_fix.reshape(1, pop.slots, 9)[0]
    x0 = M.encode(pop.parent[0], pop.axis[0], R9, pop.p_fix[0], pop.com[0], pop.w_int[0], pop.w_cpl[0], nb)
    # renumber: a topological order of the tree that visits children in reverse
    kids = {b: [c for c in range(1, nb) if pop.parent[0, c] == b] for b in range(nb)}
    order, stack = [], [0]
    while stack:
        b = stack.pop()
        order.append(b)
        stack.extend(kids[b])
    new_of = {old: new for new, old in enumerate(order)}
    par = np.array([-1] + [new_of[pop.parent[0, o]] for o in order[1:]])
    perm = np.array(order)
    x1 = M.encode(par, pop.axis[0][perm], R9[perm], pop.p_fix[0][perm], pop.com[0][perm], pop.w_int[0][perm],
                  pop.w_cpl[0][perm], nb)
    assert np.array_equal(x0, x1)
    # shift the centre of a leaf brick by 1 mm along its body's own x: only its slot's x, y, z change
    leaf = max(b for b in range(1, nb) if not kids[b])
    com = pop.com[0].copy()
    com[leaf, 0] += 0.001
    x2 = M.encode(pop.parent[0], pop.axis[0], R9, pop.p_fix[0], com, pop.w_int[0], pop.w_cpl[0], nb)
    d = np.flatnonzero(x0 != x2)
    assert 1 <= len(d) <= 3 * 6  # its own centre, and slots that swapped because of it
    assert np.isclose(np.abs(np.sort(x0[:120]) - np.sort(x2[:120])).sum(), 1 / 256.0)


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
