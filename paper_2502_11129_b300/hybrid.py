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


def hybrid_point(pop: P.Population, steps: int, gpu_factory: Callable, cpu_factory: Callable,
                 reps: int = 3) -> dict:
    """The four measurements of the paper's Sec. 6 for one population."""
    gpu_all = _Run(gpu_factory, pop)
    cpu_all = _Run(cpu_factory, pop)
    try:
        _timed(gpu_all, steps)  # captures the GPU graph for this step count
        t_gpu = [_timed(gpu_all, steps)[0] for _ in range(reps)]
        t_cpu = [_timed(cpu_all, steps)[0] for _ in range(reps)]
        f_gpu_seq = _timed(gpu_all, steps)[1]
        f_cpu_seq = _timed(cpu_all, steps)[1]
    finally:
        gpu_all.close()
        cpu_all.close()
    share = gpu_share(float(np.mean(t_cpu)), float(np.mean(t_gpu)))
    gi, ci = split(pop.n, share)
    gpu_part = _Run(gpu_factory, pop.subset(gi)) if gi.size else None
    cpu_part = _Run(cpu_factory, pop.subset(ci)) if ci.size else None
    try:
        if gpu_part is not None:
            _timed(gpu_part, steps)  # graph capture outside the timed region
        combined = []
        fit = np.zeros(pop.n, np.float32)
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
            combined.append(time.perf_counter() - t0)
    finally:
        for part in (gpu_part, cpu_part):
            if part is not None:
                part.close()
    return dict(variants=pop.n, steps=steps, seq_gpu_s=float(np.mean(t_gpu)), seq_cpu_s=float(np.mean(t_cpu)),
                naive_sum_s=float(np.mean(t_gpu) + np.mean(t_cpu)), combined_s=float(np.mean(combined)),
                combined_runs_s=combined, gpu_share=float(share), gpu_variants=int(gi.size),
                cpu_variants=int(ci.size),
                # every variant's result must not depend on where it ran
                same_as_sequential=bool(np.array_equal(fit[gi], f_gpu_seq[gi]) and
                                        np.array_equal(fit[ci], f_cpu_seq[ci])))


def main():
    from . import cpu as CP
    from . import sweeps as SW
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", choices=["box", "quadruped", "grammar"], default="grammar")
    ap.add_argument("--variants", type=int, nargs="*", default=[128, 512, 2048, 8192])
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    rows = []
    for n in a.variants:
        r = hybrid_point(SW.scene(a.scene, n), a.steps, lambda: S.Sim(), lambda: CP.CpuSim(threads=a.threads),
                         a.reps)
        r["scene"] = a.scene
        rows.append(r)
        print(json.dumps(r), flush=True)
    print("| scene | variants | seq CPU s | seq GPU s | naive sum s | combined s | GPU share |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['scene']} | {r['variants']} | {r['seq_cpu_s']:.3f} | {r['seq_gpu_s']:.3f} | "
              f"{r['naive_sum_s']:.3f} | {r['combined_s']:.3f} | {100 * r['gpu_share']:.1f} % |")


if __name__ == "__main__":
    main()
