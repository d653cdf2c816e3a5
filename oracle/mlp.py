"""FP64 oracle of the learned surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
module; it shares no code with the CUDA surrogate library.

What it computes, plainly (the paper's EA context, Sec. 1: memetic / Lamarckian
evolution of robot morphologies and controllers, where evaluations are
simulations):
  * encode   -- a robot genotype as a 128-d vector: 20 brick slots x
                (present, parent / 20, face / 5, rotation / 3, CPG weight),
                then the 19 coupling weights of bricks 2..20, zero padding;
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


def encode(parent, face, rot, w_int, w_cpl, nb) -> np.ndarray:
    """128-d encoding of one robot (arrays indexed by body, body 0 = core)."""
    x = np.zeros(IN_DIM)
    for i in range(SLOTS):
        b = i + 1
        if b < nb:
            x[5 * i + 0] = 1.0
            x[5 * i + 1] = parent[b] / 20.0
            x[5 * i + 2] = face[b] / 5.0
            x[5 * i + 3] = rot[b] / 3.0
            x[5 * i + 4] = w_int[b]
    for i in range(SLOTS - 1):
        b = i + 2
        if b < nb:
            x[100 + i] = w_cpl[b]
    return x


def encode_population(pop) -> np.ndarray:
    return np.stack([encode(pop.parent[i], pop.genome_face[i], pop.genome_rot[i], pop.w_int[i],
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
