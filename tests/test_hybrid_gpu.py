"""Hybrid CPU + GPU allocation (the paper's Sec. 6) with the real engines:
libb3sim on the GPU and libb3cpu on the host cores, run concurrently."""
import pytest

from paper_2502_11129_b300 import cpu as CP
from paper_2502_11129_b300 import hybrid as H
from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S

pytestmark = pytest.mark.gpu


def test_hybrid_point_runs_both_engines_concurrently():
    pop = P.grammar(512, seed=9)
    r = H.hybrid_point(pop, 100, lambda: S.Sim(), lambda: CP.CpuSim(), reps=1)
    print(r)
    assert r["seq_cpu_s"] > r["seq_gpu_s"]
    for mode in ("proportional", "longest-first"):
        m = r[mode]
        assert m["gpu_variants"] + m["cpu_variants"] == 512
        assert m["gpu_variants"] > m["cpu_variants"]  # the B300 is the faster device here
        assert m["same_as_sequential"] and m["combined_s"] > 0
