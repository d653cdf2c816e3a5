"""Simulation-driven evolution with surrogate pre-screening (orchestration).

The paper's setting (Sec. 1) is evolutionary robotics with memetic /
Lamarckian evolution: morphologies evolve, and each generation a local search
adapts every morphology's controller, so the number of simulations per
generation is (morphologies x controller samples).  Sec. 3 finds that physics
simulation takes over 80 % of such a run.  This module runs that loop on the
GPU simulator (libb3sim) and, optionally, lets the learned surrogate
(libb3sur) pre-screen candidate controllers so that only the most promising
are simulated.  It orchestrates the two C ABIs; every arithmetic step
(simulation, encoding, MLP, top-k) runs in their kernels.

Readings (the paper gives no EA parameters): controller local search =
Gaussian perturbation (sigma 0.1) of a morphology's CPG weights, clipped to
[-1, 1]; Lamarckian write-back = a morphology adopts its best simulated
controller if it beats the current one; morphology selection = the better
half survives, the worse half is replaced by fresh grammar robots; the
surrogate is retrained every generation on all (genotype, fitness) pairs
simulated so far and screens `screen_factor` x more candidate controllers
and `screen_morph` x more fresh morphologies than are simulated.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np

from . import population as P
from . import shard as SH
from . import sim as S
from . import surrogate as SG

# process group when launched with one process per GPU (torchrun); every rank
# runs the same EA loop with the same seeds and simulates its shard of each
# population (see shard.py)
_DIST = None
_DEVICE = 0


# A robot whose core ever moves faster than this (checked every CHECK_EVERY
# steps) has gained energy the servos cannot supply (1 N m on 0.2 kg bricks
# walks at well under 1 m/s): the evolution loop scores it 0, like a frozen
# robot.  Evolution otherwise finds controllers that trigger the rare
# energy-injecting contact configurations of the soft-contact model (the FP64
# oracle reproduces them from the same genome), and their "displacement" is a
# launch, not locomotion.
MAX_CORE_SPEED = 2.0  # m/s
CHECK_EVERY = 250


def _simulate_local(pop: P.Population, steps: int, **cfg) -> np.ndarray:
    cfg.setdefault("device", _DEVICE)
    sm = S.Sim(**cfg)
    try:
        sm.set_population(pop)
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        sm.set_state(Q, V, Sx)
        vmax = np.zeros(pop.n)
        done = 0
        while done < steps:
            k = min(CHECK_EVERY, steps - done)
            sm.step(k)
            done += k
            v = sm.read_state()[1]
            vmax = np.maximum(vmax, np.linalg.norm(v[:, :3], axis=1))
        f = sm.fitness()
        st = sm.read_state()[3]
        f[(st & 5) != 0] = 0.0  # a frozen robot earns nothing
        f[~(vmax <= MAX_CORE_SPEED)] = 0.0  # nor does a launched one
        return f.astype(np.float64)
    finally:
        sm.close()


def simulate(pop: P.Population, steps: int, **cfg) -> np.ndarray:
    """Core xy displacement of every robot after `steps` steps from rest
    (sharded over the ranks of the process group, if there is one)."""
    return SH.run_sharded(pop, lambda sub: _simulate_local(sub, steps, **cfg), _DIST)


def ranks(a):
    a = np.asarray(a, dtype=np.float64)
    order = np.argsort(a, kind="mergesort")
    r = np.empty(len(a))
    r[order] = np.arange(len(a), dtype=np.float64)
    # average ties
    sa = a[order]
    i = 0
    while i < len(a):
        j = i
        while j + 1 < len(a) and sa[j + 1] == sa[i]:
            j += 1
        if j > i:
            r[order[i:j + 1]] = 0.5 * (i + j)
        i = j + 1
    return r


def spearman(a, b) -> float:
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    return float((ra @ rb) / np.sqrt((ra @ ra) * (rb @ rb)))


def mann_whitney_greater(x, y) -> float:
    """One-sided p-value that x tends to exceed y (normal approximation with
    tie correction)."""
    n1, n2 = len(x), len(y)
    r = ranks(np.concatenate([x, y])) + 1.0
    u = r[:n1].sum() - n1 * (n1 + 1) / 2.0
    mu = n1 * n2 / 2.0
    _, counts = np.unique(np.concatenate([x, y]), return_counts=True)
    n = n1 + n2
    tie = (counts ** 3 - counts).sum() / (n * (n - 1))
    sd = np.sqrt(n1 * n2 / 12.0 * ((n + 1) - tie))
    z = (u - mu - 0.5) / sd
    from math import erfc, sqrt
    return 0.5 * erfc(z / sqrt(2.0))


def screening(n_train=50000, n_screen=65536, k=4096, steps=5000, epochs=30, batch=1024, seed=4,
              full_eval=False) -> dict:
    """Train on simulated (genotype, displacement) pairs, screen offspring,
    simulate the top k and k random ones."""
    t0 = time.perf_counter()
    train = P.grammar(n_train, seed=seed)
    f_train = simulate(train, steps)
    t_sim = time.perf_counter() - t0
    sur = SG.Surrogate(seed=seed, device=_DEVICE)
    X = sur.encode(train)
    t1 = time.perf_counter()
    loss = sur.train(X, f_train.astype(np.float32), epochs=epochs, batch=batch)
    t_train = time.perf_counter() - t1
    cand = P.grammar(n_screen, seed=seed + 1)
    t2 = time.perf_counter()
    pred = sur.predict(sur.encode(cand))
    top = sur.topk(pred, k)
    t_screen = time.perf_counter() - t2
    rng = np.random.default_rng(seed + 2)
    rnd = rng.choice(n_screen, size=k, replace=False)
    f_top = simulate(cand.subset(top), steps)
    f_rnd = simulate(cand.subset(rnd), steps)
    out = dict(n_train=n_train, n_screen=n_screen, k=k, steps=steps, epochs=epochs, train_loss=loss,
               spearman_top=spearman(pred[top], f_top), mae_top=float(np.mean(np.abs(pred[top] - f_top))),
               spearman_random=spearman(pred[rnd], f_rnd), mae_random=float(np.mean(np.abs(pred[rnd] - f_rnd))),
               mean_fitness_top=float(f_top.mean()), mean_fitness_random=float(f_rnd.mean()),
               p_top_beats_random=mann_whitney_greater(f_top, f_rnd),
               seconds_simulate_train=t_sim, seconds_train=t_train, seconds_screen=t_screen)
    if full_eval:
        f_all = simulate(cand, steps)
        out["spearman_all"] = spearman(pred, f_all)
        out["mae_all"] = float(np.mean(np.abs(pred - f_all)))
    sur.close()
    return out


@dataclasses.dataclass
class RunLog:
    best: list
    evals: list
    sims: list
    seconds: list


def _perturb(pop: P.Population, idx, rng, sigma, count) -> P.Population:
    """`count` controller variants of each robot in idx (weights + N(0, sigma),
    clipped to [-1, 1]); couplings exist only where the parent is a brick."""
    rep = np.repeat(np.asarray(idx), count)
    out = pop.subset(rep)
    nb = out.nb
    mask = np.arange(P.MAXB)[None, :] < nb[:, None]
    mask[:, 0] = False
    cpl = mask & (out.parent >= 1)
    out.w_int = np.where(mask, np.clip(out.w_int + rng.normal(0, sigma, out.w_int.shape), -1, 1), 0.0)
    out.w_cpl = np.where(cpl, np.clip(out.w_cpl + rng.normal(0, sigma, out.w_cpl.shape), -1, 1), 0.0)
    return out


def memetic(n_morph=256, n_ctrl=64, gens=30, steps=5000, sigma=0.1, surrogate=False, screen_factor=4,
            epochs=10, batch=1024, seed=5, target=None, log=print, save_best=None, screen_morph=1,
            relative=False) -> dict:
    """Lamarckian memetic loop; returns the best-fitness trace with wall time
    and the number of offspring considered (evaluations) and simulated.
    With the surrogate on, it screens screen_factor x the controller
    variants of every morphology and screen_morph x the fresh morphologies
    (1: fresh morphologies unscreened).
    relative: the network learns an offspring's fitness minus its parent's
    (the morphology's best when the offspring was drawn), from the simulated
    offspring only, so that its capacity goes to the differences between
    siblings, which is all the screening ranks; until it has data, the
    loop simulates unscreened offspring.
    save_best: path of an .npz that receives the final best robot (every
    Population field of it)."""
    if relative and screen_morph > 1:
        raise ValueError("relative targets rank siblings only: screen_morph must be 1")
    rng = np.random.default_rng(seed)
    morphs = P.grammar(n_morph, seed=seed)
    best_f = simulate(morphs, steps)
    sur = SG.Surrogate(seed=seed, device=_DEVICE) if surrogate else None
    data_X = [sur.encode(morphs)] if surrogate and not relative else []
    data_y = [best_f.copy()] if not relative else []
    trace = RunLog([float(best_f.max())], [n_morph], [n_morph], [0.0])
    t0 = time.perf_counter()
    evals = n_morph
    sims = n_morph
    reached = None
    for gen in range(gens):
        if surrogate and data_y:
            X_all = np.concatenate(data_X)
            y_all = np.concatenate(data_y).astype(np.float32)
            sur.train(X_all, y_all, epochs=epochs, batch=min(batch, len(y_all)))
            cand = _perturb(morphs, np.arange(n_morph), rng, sigma, n_ctrl * screen_factor)
            pred = sur.predict(sur.encode(cand))
            keep = []
            for m in range(n_morph):
                lo = m * n_ctrl * screen_factor
                sel = sur.topk(pred[lo:lo + n_ctrl * screen_factor], n_ctrl)
                keep.append(lo + sel)
            keep = np.concatenate(keep)
            offspring = cand.subset(keep)
            evals += cand.n
        else:
            offspring = _perturb(morphs, np.arange(n_morph), rng, sigma, n_ctrl)
            evals += offspring.n
        f = simulate(offspring, steps)
        sims += offspring.n
        if surrogate:
            data_X.append(sur.encode(offspring))
            data_y.append(f - np.repeat(best_f, n_ctrl) if relative else f)
        # Lamarckian write-back of the best controller of each morphology
        fm = f.reshape(n_morph, n_ctrl)
        arg = fm.argmax(axis=1)
        for m in range(n_morph):
            if fm[m, arg[m]] > best_f[m]:
                j = m * n_ctrl + arg[m]
                morphs.w_int[m] = offspring.w_int[j]
                morphs.w_cpl[m] = offspring.w_cpl[j]
                best_f[m] = fm[m, arg[m]]
        # morphology selection: the better half survives, fresh robots replace the rest
        order = np.argsort(-best_f, kind="stable")
        keep_m = order[: n_morph // 2]
        n_fresh = n_morph - len(keep_m)
        if surrogate and screen_morph > 1:
            # the network ranks different morphologies far better than
            # controller perturbations of one (cfg4): draw screen_morph x the
            # fresh morphologies and simulate the predicted best
            cand_m = P.grammar(n_fresh * screen_morph, seed=seed + 1000 * (gen + 1))
            evals += cand_m.n - n_fresh
            fresh = cand_m.subset(np.sort(sur.topk(sur.predict(sur.encode(cand_m)), n_fresh)))
        else:
            fresh = P.grammar(n_fresh, seed=seed + 1000 * (gen + 1))
        f_fresh = simulate(fresh, steps)
        sims += fresh.n
        evals += fresh.n
        if surrogate and not relative:
            data_X.append(sur.encode(fresh))
            data_y.append(f_fresh)
        kept = morphs.subset(keep_m)
        morphs = _concat(kept, fresh)
        best_f = np.concatenate([best_f[keep_m], f_fresh])
        el = time.perf_counter() - t0
        trace.best.append(float(best_f.max()))
        trace.evals.append(evals)
        trace.sims.append(sims)
        trace.seconds.append(el)
        if target is not None and reached is None and best_f.max() >= target:
            reached = dict(gen=gen + 1, seconds=el, evals=evals, sims=sims)
        log(f"gen {gen + 1}: best {best_f.max():.4f} evals {evals} sims {sims} {el:.1f}s")
    if sur is not None:
        sur.close()
    if save_best:
        best = morphs.subset([int(np.argmax(best_f))])
        np.savez(save_best, fitness=best_f.max(),
                 **{f.name: getattr(best, f.name) for f in dataclasses.fields(best)})
    return dict(surrogate=surrogate, best=trace.best, evals=trace.evals, sims=trace.sims, seconds=trace.seconds,
                reached=reached, final_best=trace.best[-1], evals_per_s=evals / trace.seconds[-1])


def _concat(a: P.Population, b: P.Population) -> P.Population:
    fields = {}
    for f in dataclasses.fields(a):
        va, vb = getattr(a, f.name), getattr(b, f.name)
        fields[f.name] = np.concatenate([va, vb]) if isinstance(va, np.ndarray) else va
    fields["n"] = a.n + b.n
    return P.Population(**fields)


def _init_dist():
    """One process per GPU under torchrun: device = LOCAL_RANK."""
    global _DIST, _DEVICE
    import os
    if int(os.environ.get("WORLD_SIZE", "1")) <= 1:
        return 0
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend="gloo")
    _DIST = dist
    _DEVICE = int(os.environ.get("LOCAL_RANK", "0"))
    return _DEVICE


def main():
    _init_dist()
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["screening", "memetic"], default="screening")
    ap.add_argument("--n-train", type=int, default=50000)
    ap.add_argument("--n-screen", type=int, default=65536)
    ap.add_argument("--k", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--morph", type=int, default=256)
    ap.add_argument("--ctrl", type=int, default=64)
    ap.add_argument("--gens", type=int, default=30)
    ap.add_argument("--screen-factor", type=int, default=4)
    ap.add_argument("--screen-morph", type=int, default=1)
    ap.add_argument("--relative", action="store_true", help="train the screening network on fitness minus the parent's")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--full-eval", action="store_true")
    a = ap.parse_args()
    lead = _DIST is None or _DIST.get_rank() == 0
    say = print if lead else (lambda *args, **kw: None)
    if a.mode == "screening":
        out = screening(a.n_train, a.n_screen, a.k, a.steps, a.epochs, seed=a.seed, full_eval=a.full_eval)
    else:
        plain = memetic(a.morph, a.ctrl, a.gens, a.steps, surrogate=False, seed=a.seed, log=say)
        sur = memetic(a.morph, a.ctrl, a.gens, a.steps, surrogate=True, screen_factor=a.screen_factor,
                      seed=a.seed, target=plain["final_best"], log=say, screen_morph=a.screen_morph,
                      relative=a.relative)
        out = dict(plain=plain, surrogate=sur)
    say(json.dumps(out))
    if _DIST is not None:
        _DIST.destroy_process_group()


if __name__ == "__main__":
    main()
