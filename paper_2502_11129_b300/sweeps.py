"""Scaling sweeps of the GPU simulator in the shape of the paper's benchmarks.

Sec. 4 times N variants of a scene for 1000 steps with N from 32 to 512000
(3 repetitions, 95 % confidence intervals), and Sec. 5 times 128 variants for
32 to 32768 steps; both show the GPU run time flat while the device is not
full and linear after.  This module runs the same two sweeps on this
simulator:

    python -m paper_2502_11129_b300.sweeps --sweep variants --scene box
    python -m paper_2502_11129_b300.sweeps --sweep steps --scene grammar

Scenes: ``box`` (one free 0.1 m cube per variant, the BOX-like scene),
``box_and_ball`` (a cube with one hinged ball, the BOX_AND_BALL-like scene),
``rope`` (a cube trailing a passive chain, 25 links by default: the
ARM_WITH_ROPE-like scene; ``--links`` up to 63, where chains of more than 25
links take the block-per-robot kernel), ``quadruped``, ``grammar``
(tree-grammar robots with 2..20 hinges) and ``grammar_balls`` (the same with
30 % of the modules balls).  Large populations other than ``box`` repeat a
base population of 4096 distinct robots (generating robots is host work that
the sweep does not time).

Each point: build the population and the simulator, one untimed call that
captures the CUDA graph for that step count, then 3 timed calls, each from
the same initial state: wall time of sim_step_n plus the fitness read that
waits for it.  Printed per point: mean seconds, the 95 % confidence
half-width (Student t, 2 degrees of freedom) and variant-steps/s.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import population as P
from . import sim as S

PAPER_VARIANTS = (32, 128, 256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536, 131072, 256000, 512000)
PAPER_STEPS = (32, 128, 256, 512, 1024, 2048, 4096, 8192, 16384, 32768)
# Student t quantile 0.975 with 2 degrees of freedom: the CDF there is
# 1/2 + t / (2 sqrt(2 + t^2)), so t = sqrt(2 q^2 / (1 - q^2)) with q = 0.95
T_975_DF2 = math.sqrt(2 * 0.95 ** 2 / (1 - 0.95 ** 2))
BASE_ROBOTS = 4096  # distinct robots behind large quadruped / grammar populations

_BASE = {}


_MAKERS = {
    "quadruped": lambda n, seed: P.quadrupeds(n, seed=seed),
    "grammar": lambda n, seed: P.grammar(n, seed=seed),
    "grammar_balls": lambda n, seed: P.grammar(n, seed=seed, ball_p=0.3),
    "box_and_ball": lambda n, seed: P.box_and_ball(n, seed=seed),
    "rope": lambda n, seed, links=25: P.rope(n, seed=seed, links=links),
}
SCENES = ("box",) + tuple(_MAKERS)
# simulator settings a scene runs with (a rope is a passive chain)
SCENE_CFG = {"rope": dict(actuate=0)}


def scene(name: str, n: int, seed: int = 1, links: int | None = None) -> P.Population:
    if name == "box":
        return P.boxes(n, seed=seed)
    if name not in _MAKERS:
        raise ValueError(f"unknown scene {name!r}")
    if links is not None and name != "rope":
        raise ValueError("links applies to the rope scene only")
    base_n = min(n, BASE_ROBOTS)
    key = (name, seed, links)
    if key not in _BASE or _BASE[key].n < base_n:
        extra = {} if links is None else {"links": links}
        _BASE[key] = _MAKERS[name](base_n, seed, **extra)
    base = _BASE[key]
    return base.subset(np.arange(n) % base.n)


def time_point(pop: P.Population, steps: int, reps: int = 3, **cfg) -> dict:
    sm = S.Sim(**cfg)
    try:
        sm.set_population(pop)
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        sm.set_state(Q, V, Sx)
        sm.step(steps)  # captures the graph for this step count
        sm.fitness()
        ts = []
        for _ in range(reps):
            sm.set_state(Q, V, Sx)
            t0 = time.perf_counter()
            sm.step(steps)
            sm.fitness()
            ts.append(time.perf_counter() - t0)
        c = sm.counters()
    finally:
        sm.close()
    ts = np.asarray(ts)
    mean = float(ts.mean())
    half = float(T_975_DF2 * ts.std(ddof=1) / math.sqrt(reps)) if reps > 1 else 0.0
    return dict(variants=pop.n, steps=steps, seconds=ts.tolist(), mean_s=mean, ci95_s=half,
                variant_steps_per_s=pop.n * steps / mean,
                contacts_per_variant_step=c["contacts"] / max(c["variant_steps"], 1))


def sweep(kind: str, scene_name: str, values=None, reps: int = 3, seed: int = 1, log=print,
          links: int | None = None) -> list:
    rows = []
    label = scene_name if links is None else f"{scene_name}-{links}"
    if kind == "variants":
        for n in values or PAPER_VARIANTS:
            r = time_point(scene(scene_name, n, seed, links), 1000, reps, **SCENE_CFG.get(scene_name, {}))
            r["scene"] = label
            rows.append(r)
            log(json.dumps(r))
    elif kind == "steps":
        pop = scene(scene_name, 128, seed, links)
        for s in values or PAPER_STEPS:
            r = time_point(pop, s, reps, **SCENE_CFG.get(scene_name, {}))
            r["scene"] = label
            rows.append(r)
            log(json.dumps(r))
    else:
        raise ValueError(kind)
    return rows


def table(rows) -> str:
    out = ["| scene | variants | steps | mean s | ±95 % s | variant-steps/s |", "|---|---|---|---|---|---|"]
    for r in rows:
        out.append(f"| {r['scene']} | {r['variants']} | {r['steps']} | {r['mean_s']:.4f} | {r['ci95_s']:.4f} | "
                   f"{r['variant_steps_per_s']:.3e} |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sweep", choices=["variants", "steps"], default="variants")
    ap.add_argument("--scene", choices=list(SCENES), default="box")
    ap.add_argument("--values", type=int, nargs="*")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--links", type=int, default=None, help="chain length of the rope scene (1..63)")
    a = ap.parse_args()
    rows = sweep(a.sweep, a.scene, a.values, a.reps, a.seed, links=a.links)
    print(table(rows))


if __name__ == "__main__":
    main()
