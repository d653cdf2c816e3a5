"""FP64 oracle of the learned surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
module; it shares no code with the CUDA surrogate library.

What it computes, plainly (the paper's EA context, Sec. 1: memetic / Lamarckian
evolution of robot morphologies and controllers, where evaluations are
simulations):
  * encode   -- a robot as a 128-d vector: its bricks' zero-pose geometry
                and controller weights, 20 slots of 6 (centre x, y, z in the
                core frame in millimetres / 256, hinge-axis code / 3, CPG
                weight, coupling weight to the parent hinge), bricks ordered
                by centre (z, then x, then y), zero padding;
  * forward  -- y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 on BF16-rounded
                weights and inputs, FP64 arithmetic;
  * loss     -- mean squared error on standardised targets;
  * backward -- analytic gradients of the loss (chain rule, ReLU mask);
  * adam     -- Kingma & Ba 2015, Algorithm 1 (bias-corrected moments);
  * topk     -- indices of the k largest scores, ties to the lower index;
  * spearman -- Pearson correlation of average ranks.
Pins (tests/test_surrogate_oracle.py): central finite differences of the loss
for every gradient entry on a small network; a hand-worked forward pass; the
Adam update against the algorithm's first step written out; encoding of a
hand-built genotype; top-k against a full sort; Spearman against a library
routine and on monotone transforms (exactly 1).
"""
from __future__ import annotations

import numpy as np

IN_DIM = 128
SLOTS = 20


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def zero_pose_mm(parent, R_fix, p_fix, com, nb):
    """Box centres and rotations of every body at zero hinge angles, in the
    core frame, on the integer millimetre lattice: joint rotations rounded
    to their integer entries, offsets to whole millimetres (exact for the
    lattice-built robots).  Parents precede children."""
    R = [np.eye(3, dtype=np.int64)]
    o = [np.zeros(3, np.int64)]
    c = [np.rint(np.asarray(com[0], np.float64) * 1000.0).astype(np.int64)]
    for b in range(1, nb):
        Rf = np.rint(np.asarray(R_fix[b], np.float64)).astype(np.int64).reshape(3, 3)
        pf = np.rint(np.asarray(p_fix[b], np.float64) * 1000.0).astype(np.int64)
        cb = np.rint(np.asarray(com[b], np.float64) * 1000.0).astype(np.int64)
        Rp, op = R[parent[b]], o[parent[b]]
        R.append(Rp @ Rf)
        o.append(op + Rp @ pf)
        c.append(o[b] + R[b] @ cb)
    return R, c


def encode(parent, axis, R_fix, p_fix, com, w_int, w_cpl, nb) -> np.ndarray:
    """128-d encoding of one robot (arrays indexed by body, body 0 = core)."""
    R, c = zero_pose_mm(parent, R_fix, p_fix, com, nb)
    rows = []
    for b in range(1, nb):
        a = R[b][:, int(axis[b])]  # hinge axis in the core frame: a signed unit vector
        code = int(np.argmax(np.abs(a))) + 1
        cpl = w_cpl[b] if parent[b] >= 1 else 0.0
        rows.append(((int(c[b][2]), int(c[b][0]), int(c[b][1])),
                     [c[b][0] / 256.0, c[b][1] / 256.0, c[b][2] / 256.0, code / 3.0, float(w_int[b]), float(cpl)]))
    rows.sort(key=lambda r: r[0])
    x = np.zeros(IN_DIM)
    for i, (_, f) in enumerate(rows[:SLOTS]):
        x[6 * i:6 * i + 6] = f
    return x


def encode_population(pop) -> np.ndarray:
    R9 = pop.R_fix.reshape(pop.n, pop.slots, 9)
    return np.stack([encode(pop.parent[i], pop.axis[i], R9[i], pop.p_fix[i], pop.com[i], pop.w_int[i],
                            pop.w_cpl[i], int(pop.nb[i])) for i in range(pop.n)])


def init_params(rng, hidden=256, in_dim=IN_DIM):
    """He-uniform weights, zero biases (float64 master copies)."""
    def he(n_out, n_in):
        lim = np.sqrt(6.0 / n_in)
        return rng.uniform(-lim, lim, size=(n_out, n_in))
    return dict(W1=he(hidden, in_dim), b1=np.zeros(hidden), W2=he(hidden, hidden), b2=np.zeros(hidden),
                W3=he(1, hidden), b3=np.zeros(1))


def forward(p, X):
    """Returns y (n,) and the cache for backward.  X and weights BF16-rounded."""
    Xb = bf16_round(X)
    W1, W2, W3 = bf16_round(p["W1"]), bf16_round(p["W2"]), bf16_round(p["W3"])
    z1 = Xb @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + p["b3"]
    return y[:, 0], dict(X=Xb, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, W3=W3)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.mean((y - t) ** 2))


def backward(p, X, t):
    """Analytic gradients of the mean squared error with respect to all
    parameters (taken at the BF16-rounded weights)."""
    y, c = forward(p, X)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                     # (n,)
    g = {}
    g["W3"] = dy[None, :] @ c["h2"]            # (1, H)
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] @ c["W3"]                # (n, H)
    dz2 = dh2 * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ c["W2"]
    dz1 = dh1 * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(axis=0)
    return g, float(np.mean((y - t) ** 2))


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1-based step count); returns new p, m, v."""
    p2, m2, v2 = {}, {}, {}
    for k in p:
        m2[k] = b1 * m[k] + (1 - b1) * g[k]
        v2[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m2[k] / (1 - b1 ** t)
        vh = v2[k] / (1 - b2 ** t)
        p2[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def topk(scores, k):
    """Indices of the k largest scores, ties to the lower index, ordered by
    descending score (then ascending index)."""
    s = np.asarray(scores, dtype=np.float64)
    order = np.lexsort((np.arange(len(s)), -s))
    return order[:k]


def average_ranks(a):
    a = np.asarray(a, dtype=np.float64)
    order = np.argsort(a, kind="mergesort")
    ranks = np.empty(len(a))
    i = 0
    while i < len(a):
        j = i
        while j + 1 < len(a) and a[order[j + 1]] == a[order[i]]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1.0
        i = j + 1
    return ranks


def spearman(a, b):
    ra, rb = average_ranks(a), average_ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra @ rb) / np.sqrt((ra @ ra) * (rb @ rb)))
