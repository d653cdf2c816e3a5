"""Surrogate-screened evolution on the GPU (small sizes).

Gain test: offspring chosen by the trained surrogate simulate to higher
fitness than offspring chosen at random (one-sided Mann-Whitney p < 0.01).
The memetic loop runs end to end with the surrogate on and off, and with
relative targets.
"""
import numpy as np
import pytest

from paper_2502_11129_b300 import evolve as E

pytestmark = pytest.mark.gpu


def test_surrogate_top_k_beats_random_offspring():
    r = E.screening(n_train=8192, n_screen=16384, k=1024, steps=1500, epochs=30, batch=512, seed=11)
    print(r)
    assert r["p_top_beats_random"] < 0.01, r
    assert r["mean_fitness_top"] > r["mean_fitness_random"]
    assert r["spearman_random"] > 0.2, r


def test_memetic_loop_runs_with_and_without_surrogate():
    plain = E.memetic(n_morph=16, n_ctrl=8, gens=2, steps=300, surrogate=False, seed=3, log=lambda *a: None)
    sur = E.memetic(n_morph=16, n_ctrl=8, gens=2, steps=300, surrogate=True, screen_factor=4, seed=3,
                    log=lambda *a: None)
    assert len(plain["best"]) == 3 and len(sur["best"]) == 3
    assert plain["best"][-1] >= plain["best"][0]  # Lamarckian write-back never loses the best
    assert sur["evals"][-1] > plain["evals"][-1]  # the surrogate considers more offspring per simulation
    assert sur["sims"][-1] == plain["sims"][-1]


def test_memetic_loop_with_relative_targets():
    """Relative targets: the first generation has no training data and
    simulates unscreened offspring drawn as the plain loop draws them (the
    same best); later generations screen."""
    plain = E.memetic(n_morph=16, n_ctrl=8, gens=3, steps=300, surrogate=False, seed=4, log=lambda *a: None)
    rel = E.memetic(n_morph=16, n_ctrl=8, gens=3, steps=300, surrogate=True, screen_factor=4, seed=4,
                    relative=True, log=lambda *a: None)
    assert rel["best"][1] == plain["best"][1]
    assert rel["evals"][1] == plain["evals"][1]
    assert rel["evals"][-1] > plain["evals"][-1] and rel["sims"][-1] == plain["sims"][-1]
    assert rel["best"][-1] >= rel["best"][0]


def test_rank_helpers_match_library():
    import scipy.stats
    rng = np.random.default_rng(0)
    a = rng.normal(size=200)
    b = a + rng.normal(size=200)
    b[::5] = b[1]
    assert abs(E.spearman(a, b) - scipy.stats.spearmanr(a, b).statistic) < 1e-12
    x, y = a[:100] + 0.5, a[100:]
    p = E.mann_whitney_greater(x, y)
    ref = scipy.stats.mannwhitneyu(x, y, alternative="greater", method="asymptotic").pvalue
    assert abs(p - ref) < 1e-6
