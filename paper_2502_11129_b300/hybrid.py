"""Hybrid CPU + GPU allocation of variants (the paper's Sec. 6).

The paper's strategy, step by step:
  1. initial benchmarking -- run the variants sequentially on the CPU engine
     and on the GPU and record both wall times;
  2. dynamic allocation -- split the variants between the two devices in
     proportion to their measured speed (the reversed time ratio): the GPU
     takes t_cpu / (t_cpu + t_gpu) of them;
  3. concurrent execution -- run both shares at the same time (the GPU
     simulator is asynchronous: its graph is launched first, then the host
     threads run the CPU share) and record the wall clock;
  4. report Sequential CPU, Sequential GPU, Naive Sum (t_cpu + t_gpu),
     Combined (the concurrent wall clock) and the GPU's share of variants.

A second allocation, "longest-first", departs from the paper on purpose.
A GPU step launch lasts as long as its slowest robot (one warp per robot, all
robots in flight at once), so removing robots from the GPU shortens its run
only if the heaviest ones go; and one host core steps a heavy robot several
times faster than one GPU warp does.  So the CPU takes the robots with the
largest measured GPU cost, as many as keep the predicted CPU time (longest-
processing-time-first over its worker threads, per-robot CPU times from the
sequential run) below the predicted GPU time of the rest (the sequential GPU
time scaled by the larger of the heaviest remaining robot's cost relative to
the heaviest overall and the fraction of robots remaining).

Engines are passed in as factories returning objects with the Sim / CpuSim
interface (set_population, set_state, step, fitness, read_state, close), so
the allocation logic is the same whichever engines are paired.  The GPU side
is sim.Sim (libb3sim) and the CPU side cpu.CpuSim (libb3cpu); neither falls
back to the other.

    python -m paper_2502_11129_b300.hybrid --scene grammar --variants 128 512 2048 8192
"""
from __future__ import annotations

import argparse
import json
import time
from typing import Callable

import numpy as np

from . import population as P
from . import sim as S


def gpu_share(t_cpu: float, t_gpu: float) -> float:
    """Fraction of the variants for the GPU: speeds are n/t, so the GPU gets
    (n/t_gpu) / (n/t_gpu + n/t_cpu) = t_cpu / (t_cpu + t_gpu)."""
    if not (t_cpu >= 0 and t_gpu >= 0) or t_cpu + t_gpu <= 0:
        raise ValueError("times must be non-negative and not both zero")
    return t_cpu / (t_cpu + t_gpu)


def split(n: int, share: float) -> tuple[np.ndarray, np.ndarray]:
    """Variants [0, n_gpu) to the GPU and the rest to the CPU, n_gpu the
    nearest integer to share * n."""
    n_gpu = int(min(n, max(0, round(share * n))))
    return np.arange(n_gpu), np.arange(n_gpu, n)


def longest_first_split(gpu_cost, cpu_seconds, t_gpu: float, workers: int):
    """(gpu indices, cpu indices, predicted seconds): the CPU takes the k
    robots of largest GPU cost, k minimising max(predicted CPU time,
    predicted GPU time) (see the module docstring)."""
    import heapq
    g = np.asarray(gpu_cost, dtype=np.float64)
    c = np.asarray(cpu_seconds, dtype=np.float64)
    n = g.size
    order = np.argsort(-g, kind="stable")
    gmax = max(g[order[0]], 1e-30) if n else 1.0
    loads = [0.0] * max(1, workers)
    best_k, best_t, cpu_t = 0, t_gpu, 0.0
    for k in range(1, n + 1):
        lo = heapq.heappop(loads)  # longest remaining job to the least-loaded worker
        heapq.heappush(loads, lo + c[order[k - 1]])
        cpu_t = max(cpu_t, lo + c[order[k - 1]])
        gpu_t = t_gpu * max(g[order[k]] / gmax, (n - k) / n) if k < n else 0.0
        t = max(cpu_t, gpu_t)
        if t < best_t:
            best_k, best_t = k, t
        if cpu_t >= best_t:
            break
    return np.sort(order[best_k:]), np.sort(order[:best_k]), best_t


class _Run:
    """One engine with a population loaded and its start state kept."""

    def __init__(self, factory: Callable, pop: P.Population):
        self.eng = factory()
        self.pop = pop
        self.eng.set_population(pop)
        self.rows = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))

    def reset(self):
        self.eng.set_state(*self.rows)

    def close(self):
        self.eng.close()


def _timed(run: _Run, steps: int) -> tuple[float, np.ndarray]:
    run.reset()
    t0 = time.perf_counter()
    run.eng.step(steps)
    f = run.eng.fitness()  # waits for the engine
    return time.perf_counter() - t0, f


def _concurrent(pop, steps, gi, ci, gpu_factory, cpu_factory, reps):
    """Wall clock of the GPU share and the CPU share run at the same time."""
    gpu_part = _Run(gpu_factory, pop.subset(gi)) if gi.size else None
    cpu_part = _Run(cpu_factory, pop.subset(ci)) if ci.size else None
    fit = np.zeros(pop.n, np.float32)
    try:
        # one untimed concurrent run: graph capture, host threads and work spaces warm
        for part in (gpu_part, cpu_part):
            if part is not None:
                part.reset()
        if gpu_part is not None:
            gpu_part.eng.step(steps)
        if cpu_part is not None:
            cpu_part.eng.step(steps)
            cpu_part.eng.fitness()
        if gpu_part is not None:
            gpu_part.eng.fitness()
        walls = []
        for _ in range(reps):
            for part in (gpu_part, cpu_part):
                if part is not None:
                    part.reset()
            t0 = time.perf_counter()
            if gpu_part is not None:
                gpu_part.eng.step(steps)  # asynchronous: the GPU works while the host threads run
            if cpu_part is not None:
                cpu_part.eng.step(steps)
                fit[ci] = cpu_part.eng.fitness()
            if gpu_part is not None:
                fit[gi] = gpu_part.eng.fitness()
            walls.append(time.perf_counter() - t0)
    finally:
        for part in (gpu_part, cpu_part):
            if part is not None:
                part.close()
    return walls, fit


def _cost(eng):
    """Per-robot cost of the engine's last run (GPU cycles per step, or host seconds)."""
    return eng.robot_cost() if hasattr(eng, "robot_cost") else eng.robot_seconds()


def hybrid_point(pop: P.Population, steps: int, gpu_factory: Callable, cpu_factory: Callable,
                 reps: int = 3, modes=("proportional", "longest-first")) -> dict:
    """The paper's Sec. 6 measurements for one population, for each
    allocation mode: sequential CPU and GPU, naive sum, combined."""
    gpu_all = _Run(gpu_factory, pop)
    cpu_all = _Run(cpu_factory, pop)
    try:
        _timed(gpu_all, steps)  # captures the GPU graph for this step count
        t_gpu = [_timed(gpu_all, steps)[0] for _ in range(reps)]
        t_cpu = [_timed(cpu_all, steps)[0] for _ in range(reps)]
        f_gpu_seq = _timed(gpu_all, steps)[1]
        g_cost = _cost(gpu_all.eng)
        f_cpu_seq = _timed(cpu_all, steps)[1]
        c_sec = cpu_all.eng.robot_seconds()
        workers = getattr(cpu_all.eng, "threads", 1)
    finally:
        gpu_all.close()
        cpu_all.close()
    tg, tc = float(np.mean(t_gpu)), float(np.mean(t_cpu))
    out = dict(variants=pop.n, steps=steps, seq_gpu_s=tg, seq_cpu_s=tc, naive_sum_s=tg + tc, cpu_workers=workers)
    for mode in modes:
        if mode == "proportional":
            share = gpu_share(tc, tg)
            gi, ci = split(pop.n, share)
            pred = None
        elif mode == "longest-first":
            gi, ci, pred = longest_first_split(g_cost, c_sec, tg, workers)
        else:
            raise ValueError(mode)
        walls, fit = _concurrent(pop, steps, gi, ci, gpu_factory, cpu_factory, reps)
        out[mode] = dict(combined_s=float(np.mean(walls)), combined_runs_s=walls, gpu_variants=int(gi.size),
                         cpu_variants=int(ci.size), gpu_share=gi.size / pop.n, predicted_s=pred,
                         # every variant's result must not depend on where it ran
                         same_as_sequential=bool(np.array_equal(fit[gi], f_gpu_seq[gi]) and
                                                 np.array_equal(fit[ci], f_cpu_seq[ci])))
    return out


def main():
    from . import cpu as CP
    from . import sweeps as SW
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", choices=list(SW.SCENES), default="grammar")
    ap.add_argument("--variants", type=int, nargs="*", default=[128, 512, 2048, 8192])
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    rows = []
    for n in a.variants:
        cfg = SW.SCENE_CFG.get(a.scene, {})
        r = hybrid_point(SW.scene(a.scene, n), a.steps, lambda: S.Sim(**cfg),
                         lambda: CP.CpuSim(threads=a.threads, **cfg), a.reps)
        r["scene"] = a.scene
        rows.append(r)
        print(json.dumps(r), flush=True)
    print("| scene | variants | seq CPU s | seq GPU s | naive sum s | combined s (proportional, GPU share) |"
          " combined s (longest-first, GPU share) |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        p, l = r["proportional"], r["longest-first"]
        print(f"| {r['scene']} | {r['variants']} | {r['seq_cpu_s']:.3f} | {r['seq_gpu_s']:.3f} | "
              f"{r['naive_sum_s']:.3f} | {p['combined_s']:.3f} ({100 * p['gpu_share']:.1f} %) | "
              f"{l['combined_s']:.3f} ({100 * l['gpu_share']:.1f} %) |")


if __name__ == "__main__":
    main()
