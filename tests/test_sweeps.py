"""Sweep harness: host logic on the CPU, one tiny sweep on the GPU."""
import numpy as np
import pytest

from paper_2502_11129_b300 import sweeps as SW


def test_scene_sizes_and_tiling(monkeypatch):
    b = SW.scene("box", 100)
    assert b.n == 100 and np.all(b.nb == 1)
    monkeypatch.setattr(SW, "BASE_ROBOTS", 64)
    g = SW.scene("grammar", 130, seed=5)
    base = SW.scene("grammar", 64, seed=5)
    assert g.n == 130
    # large populations repeat the base robots in order
    assert np.array_equal(g.nb[:64], base.nb[:64]) and np.array_equal(g.nb[64:128], base.nb[:64])
    with pytest.raises(ValueError):
        SW.scene("humanoid", 4)
    bb = SW.scene("box_and_ball", 8, seed=2)
    assert np.all(bb.nb == 2) and np.all(bb.geom[:, 1] == 1) and np.all(bb.geom[:, 0] == 0)
    r = SW.scene("rope", 3)
    assert np.all(r.nb == 26) and SW.SCENE_CFG["rope"] == dict(actuate=0)
    r63 = SW.scene("rope", 3, links=63)
    assert np.all(r63.nb == 64) and r63.slots == 64
    with pytest.raises(ValueError):
        SW.scene("grammar", 3, links=40)
    gb = SW.scene("grammar_balls", 40)
    assert (gb.geom == 1).any()
    # a ball is always a leaf
    for i in range(gb.n):
        for b in range(1, int(gb.nb[i])):
            if gb.geom[i, b] == 1:
                assert not (gb.parent[i, :gb.nb[i]] == b).any()


def test_t_quantile_and_table():
    import scipy.stats
    assert abs(SW.T_975_DF2 - scipy.stats.t.ppf(0.975, 2)) < 1e-9
    rows = [dict(scene="box", variants=32, steps=1000, mean_s=0.01, ci95_s=0.001, variant_steps_per_s=3.2e6)]
    assert "| box | 32 | 1000 | 0.0100 | 0.0010 | 3.200e+06 |" in SW.table(rows)


@pytest.mark.gpu
def test_tiny_sweeps_run_on_the_gpu():
    rows = SW.sweep("variants", "box", values=[32, 64], reps=2, log=lambda *a: None)
    assert [r["variants"] for r in rows] == [32, 64]
    assert all(r["mean_s"] > 0 and len(r["seconds"]) == 2 for r in rows)
    rows = SW.sweep("steps", "grammar", values=[32, 64], reps=2, log=lambda *a: None)
    assert [r["steps"] for r in rows] == [32, 64]
    for name in ("box_and_ball", "rope", "grammar_balls"):
        rows = SW.sweep("variants", name, values=[32], reps=2, log=lambda *a: None)
        assert rows[0]["mean_s"] > 0
