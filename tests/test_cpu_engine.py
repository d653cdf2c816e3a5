"""Host (CPU) engine (libb3cpu, the CPU side of the hybrid allocation) vs the
FP64 oracle, and the hybrid allocation logic -- all on the CPU.

Same bars as the GPU path (tests/parity.py): one step from identical
FP32-rounded states, every robot against the closest valid outcome of the
oracle's step, |dx| / max(|x_ref|, 1) within 1e-5 where FP32 arithmetic meets
that on every robot of the states (the oracle's FP32 build), else no worse
than that FP32 yardstick; contact-free flight within 1e-4 m over 200 steps
(or within twice FP32 arithmetic's own drift, where that exceeds 1e-4 m).
"""
import os

import numpy as np
import pytest

from paper_2502_11129_b300 import cpu as CP
from paper_2502_11129_b300 import hybrid as H
from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S
from tests import parity as PR

TOL = PR.TOL_STEP


def oracle():
    from oracle import oracle as O
    return O


def _one_step(pop, q, v, s, **cfg):
    pop32 = pop.as_float32()
    Q, V, Sx = S.state_rows(pop32, q, v, s)
    cs = CP.CpuSim(**cfg)
    cs.set_population(pop32)
    cs.set_state(Q, V, Sx)
    cs.step(1)
    gq, gv, gs, gst = cs.read_state()
    cs.close()
    prm = PR.oracle_params(**cfg)
    r = PR.one_step_errors(pop32, Q, V, Sx, gq, gv, gs, prm)
    y = PR.fp32_yardstick(pop32, Q, V, Sx, prm)
    return r, y, gst


def _check(name, r, y):
    fails = PR.parity_failures(r, y)
    msg = r.summary(name) + " | fp32 " + y.summary("yardstick") + " | " + "; ".join(fails)
    print(msg)
    assert not fails, msg


def test_one_step_boxes_quadrupeds_grammar():
    pop = P.boxes(48, seed=1)
    q = pop.q0.copy()
    q[:24, 2] = np.random.default_rng(0).uniform(0.03, 0.08, 24)
    r, y, gst = _one_step(pop, q, pop.v0, np.zeros((48, 64)))
    _check("boxes", r, y)
    assert np.array_equal(r.status_ref, gst)
    pop = P.quadrupeds(48, seed=2)
    q, v, s = P.random_state(pop, seed=5)
    q[:, 2] = np.random.default_rng(1).uniform(0.03, 0.09, pop.n)
    _check("quadrupeds", *_one_step(pop, q, v, s)[:2])
    pop = P.grammar(96, seed=3)
    q, v, s = P.random_state(pop, seed=7)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(2).uniform(-0.04, 0.0, pop.n)
    _check("grammar", *_one_step(pop, q, v, s)[:2])


def test_one_step_largest_robots_and_the_contact_cap():
    # 26 bodies in random poses: many lattice-aligned bricks sit in exact
    # separating-axis ties, compared with the closest valid outcome
    pop = P.grammar(36, seed=51, hinges=(25, 25))
    q, v, s = P.random_state(pop, seed=52)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(53).uniform(-0.03, 0.0, pop.n)
    _check("grammar-26-bodies", *_one_step(pop, q, v, s)[:2])
    pop = P.grammar(48, seed=61)
    q, v, s = P.random_state(pop, seed=62, angle=0.3)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(63).uniform(-0.045, -0.005, pop.n)
    r, y, gst = _one_step(pop, q, v, s, contact_cap=6)
    _check("cap-6", r, y)
    assert ((gst & S.ST_OVERFLOW) != 0).sum() >= 10
    assert np.array_equal((gst & S.ST_OVERFLOW) != 0, (r.status_ref & S.ST_OVERFLOW) != 0)


def test_one_step_settled_grammar_states():
    O = oracle()
    pop = P.grammar(48, seed=13).as_float32()
    q, v, s, st, _ = O.run_population(pop, pop.q0, pop.v0, P.cpg_initial(pop), 300,
                                      threads=len(os.sched_getaffinity(0)))
    _check("grammar-settled", *_one_step(pop, q, v, s)[:2])


def test_contact_free_flight_200_steps():
    O = oracle()
    pop = P.lift(P.grammar(32, seed=3), 1.0).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    cs = CP.CpuSim(box_box=0)
    cs.set_population(pop)
    cs.set_state(Q, V, Sx)
    cs.step(200)
    gq = cs.read_state()[0]
    oq, _, _, _, _ = O.run_population(pop, Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64),
                                      200, prm=O.default_params(box_box=0), threads=2)
    assert np.abs(gq[:, :3] - oq[:, :3]).max() <= 1e-4


def test_threads_do_not_change_results_and_frozen_robots_stay_put():
    pop = P.grammar(40, seed=21).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    V[7, 9] = np.nan
    out = []
    for th in (1, 3):
        cs = CP.CpuSim(threads=th)
        cs.set_population(pop)
        cs.set_state(Q, V, Sx)
        cs.step(30)
        out.append(cs.read_state())
        cs.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)
    q, v, s, st = out[0]
    assert st[7] & S.ST_NONFINITE and np.array_equal(q[7], Q[7])
    assert np.all(st[np.arange(40) != 7] & 5 == 0)


def test_abi_errors():
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        CP.CpuSim(pgs_iters=0)
    cs = CP.CpuSim()
    with pytest.raises(S.SimError, match="SIM_ESTATE"):
        cs.step(1)
    bad = P.quadrupeds(2)
    bad.parent[1, 3] = 5
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        cs.set_population(bad)
    cs.set_population(P.quadrupeds(2))
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        cs.read_state(first=1, count=5)


def test_hybrid_share_split_and_concurrent_run_on_two_host_engines():
    assert H.gpu_share(3.0, 1.0) == 0.75 and H.gpu_share(0.0, 2.0) == 0.0
    with pytest.raises(ValueError):
        H.gpu_share(0.0, 0.0)
    g, c = H.split(10, 0.75)
    assert list(g) == list(range(8)) and list(c) == [8, 9]
    pop = P.grammar(24, seed=5)
    r = H.hybrid_point(pop, 20, lambda: CP.CpuSim(threads=2), lambda: CP.CpuSim(threads=1), reps=1)
    for mode in ("proportional", "longest-first"):
        assert r[mode]["gpu_variants"] + r[mode]["cpu_variants"] == 24
        assert r[mode]["same_as_sequential"]
    assert abs(r["naive_sum_s"] - (r["seq_gpu_s"] + r["seq_cpu_s"])) < 1e-12


def test_longest_first_split_takes_the_critical_robots():
    # GPU time set by its heaviest robot (costs 10, 9, then 1s); two CPU
    # workers step a robot in 0.1 s each.  Taking k robots: CPU ceil(k/2) *
    # 0.1 s, GPU max(cost of robot k / 10, (8 - k) / 8) s; the best is k = 6
    # (CPU 0.3 s, GPU max(0.1, 0.25) s)
    g = np.array([10.0, 9.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    c = np.full(8, 0.1)
    gi, ci, t = H.longest_first_split(g, c, t_gpu=1.0, workers=2)
    assert list(ci) == [0, 1, 2, 3, 4, 5] and list(gi) == [6, 7]
    assert abs(t - 0.3) < 1e-12
    # the heaviest robots go first: with one fast worker only two fit
    gi, ci, t = H.longest_first_split(g, np.array([0.5, 0.5, 1, 1, 1, 1, 1, 1.0]), t_gpu=1.0, workers=1)
    assert list(ci) == [0] and abs(t - 0.9) < 1e-12
    # a slow CPU takes nothing
    gi, ci, t = H.longest_first_split(g, np.full(8, 5.0), t_gpu=1.0, workers=2)
    assert ci.size == 0 and t == 1.0


def _sphere_contact_kinds(pop, q):
    """Oracle contact counts by kind over a population's states: sphere/plane,
    sphere/box and sphere/sphere."""
    O = oracle()
    pop32 = pop.as_float32()
    kinds = np.zeros(3, int)
    for i in range(pop.n):
        m = O.model_from_population(pop32, i)
        c = O.contacts(m, np.asarray(q[i, :O.nq(m)], np.float64))
        for a, b in zip(c["a"], c["b"]):
            ga = m.geom[a]
            gb = m.geom[b] if b >= 0 else -1
            if b < 0 and ga == 1:
                kinds[0] += 1
            elif b >= 0 and ga + gb == 1:
                kinds[1] += 1
            elif b >= 0 and ga == 1 and gb == 1:
                kinds[2] += 1
    return kinds


def test_one_step_ball_modules_box_and_ball_and_ropes():
    """Sphere geometry (ball modules on grammar robots, a cube with a ball)
    and the longest chains (ropes of 25 links, passive) against the oracle,
    one step from random states pushed into the ground."""
    pop = P.grammar(96, seed=81, ball_p=0.4)
    q, v, s = P.random_state(pop, seed=82, angle=1.0)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(83).uniform(-0.05, 0.0, pop.n)
    kinds = _sphere_contact_kinds(pop, q)
    assert kinds.min() >= 5, kinds
    _check("ball-modules", *_one_step(pop, q, v, s)[:2])
    pop = P.box_and_ball(48, seed=84)
    q, v, s = P.random_state(pop, seed=85)
    q[:, 2] = np.random.default_rng(86).uniform(0.03, 0.12, pop.n)
    _check("box-and-ball", *_one_step(pop, q, v, s)[:2])


def fp32_flight_bar(pop, Q, V, Sx, prm, steps=200):
    """The contact-free bar of a population lifted into the air: 1e-4 m of
    core position over ``steps`` steps, or twice the drift of the oracle's own
    FP32 build from the FP64 oracle where that exceeds 1e-4 m (long chains,
    cond(M) ~ 1e5, amplify FP32 rounding step after step)."""
    from oracle import oracle32 as O32
    O = oracle()
    oq = O.run_population(pop, Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64), steps, prm=prm,
                          threads=PR.ncores())[0]
    fq = O32.run_population(pop, Q, V, Sx, steps, prm=prm, threads=PR.ncores())[0]
    drift = np.abs(fq[:, :3] - oq[:, :3]).max()
    return (1e-4 if drift <= 1e-4 else 2.0 * drift), drift


def test_one_step_ropes_against_the_fp32_yardstick():
    """Ropes of 10 and 25 links (passive), one step from random states
    pushed into the ground, against the oracle: cond(M) reaches ~1e5 on 25
    links, where FP32 arithmetic alone misses 1e-5 on most robots, so the bar
    is the FP32 yardstick's."""
    for links in (10, 25):
        pop = P.rope(24, seed=87, links=links)
        q, v, s = P.random_state(pop, seed=88, angle=0.4)
        q[:, 2] = pop.q0[:, 2] + np.random.default_rng(89).uniform(-0.04, 0.0, pop.n)
        _check(f"rope-{links}", *_one_step(pop, q, v, s, actuate=0)[:2])


def test_ropes_contact_free_and_contact_rich():
    """Lifted ropes with the servos on, 200 contact-free steps: core within
    1e-4 m of the oracle, or within twice the FP32 yardstick's own drift where
    that exceeds 1e-4 m (25 links: cond(M) ~ 1e5 amplifies FP32 rounding step
    after step).  Dropped passive 25-link ropes are chaotic and held to the
    contact-rich bar: population-mean fitness within 2 % after 2000 steps."""
    O = oracle()
    nt = max(1, len(os.sched_getaffinity(0)))
    for links in (10, 25):
        pop = P.lift(P.rope(32, seed=91, links=links), 1.0).as_float32()
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        bound, drift = fp32_flight_bar(pop, Q, V, Sx, O.default_params(box_box=0))
        cs = CP.CpuSim(box_box=0)
        cs.set_population(pop)
        cs.set_state(Q, V, Sx)
        prm = O.default_params(box_box=0)
        oq, ov, os_ = Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64)
        worst = 0.0
        for _ in range(4):
            cs.step(50)
            oq, ov, os_, _, _ = O.run_population(pop, oq, ov, os_, 50, prm=prm, threads=nt)
            worst = max(worst, np.abs(cs.read_state()[0][:, :3] - oq[:, :3]).max())
        cs.close()
        print(f"rope-{links} lifted: worst core error {worst:.3g} m, fp32 yardstick drift {drift:.3g} m")
        assert worst <= bound, (links, worst, drift)
    pop = P.rope(48, seed=92).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    cs = CP.CpuSim(actuate=0)
    cs.set_population(pop)
    cs.set_state(Q, V, Sx)
    cs.step(2000)
    gf, st = cs.fitness(), cs.read_state()[3]
    cs.close()
    oq, _, _, ost, _ = O.run_population(pop, pop.q0, pop.v0, P.cpg_initial(pop)[:, :2 * O.MAXB], 2000,
                                        prm=O.default_params(actuate=0), threads=nt)
    of = O.fitness(pop.q0, oq)
    assert (st & 5).sum() == 0 and (ost & 5).sum() == 0
    assert abs(gf.mean() - of.mean()) <= 0.02 * of.mean(), (gf.mean(), of.mean())


def test_rolling_ball_closed_form():
    """A free ball on a 20-degree incline (tilted gravity, mu = 0.5) rolls
    without slipping: acceleration (5/7) g sin(a), v = omega r."""
    G, a, r = 9.81, np.radians(20.0), 0.05
    pop = P.boxes(4, seed=3).as_float32()
    pop.geom[:, 0] = P.GEOM_SPHERE
    pop.half[:, 0] = r
    pop.mass[:, 0] = 0.5
    q = np.zeros((4, 7))
    q[:, 2] = r - 1e-4
    q[:, 3] = 1.0
    Q, V, Sx = S.state_rows(pop, q, np.zeros((4, 6)), np.zeros((4, 64)))
    cs = CP.CpuSim(mu=0.5, gravity=(G * np.sin(a), 0.0, -G * np.cos(a)))
    cs.set_population(pop)
    cs.set_state(Q, V, Sx)
    cs.step(100)
    v0 = cs.read_state()[1][:, 0].copy()
    cs.step(400)
    _, v, _, st = cs.read_state()
    cs.close()
    assert (st & 5).sum() == 0
    acc = (v[:, 0] - v0) / (400 * 0.002)
    assert np.abs(acc - 5.0 / 7.0 * G * np.sin(a)).max() < 0.01 * G * np.sin(a)
    assert np.abs(v[:, 0] - v[:, 4] * r).max() < 0.01 * np.abs(v[:, 0]).min()


def test_one_step_single_free_bodies():
    """Robots that are one free body (cubes, balls) take the one-body closed
    form of the step: tumbling cubes pressed into the ground (1-8 vertices,
    gyroscopic torque), the same with a contact cap of 3, and free balls,
    each against the oracle."""
    pop = P.boxes(64, seed=7, vel_sigma=2.0)
    rng = np.random.default_rng(8)
    q = pop.q0.copy()
    q[:, 2] = rng.uniform(0.0, 0.09, pop.n)
    r, y, gst = _one_step(pop, q, pop.v0, np.zeros((pop.n, 64)))
    _check("free-cubes", r, y)
    assert np.array_equal(r.status_ref, gst)
    r, y, gst = _one_step(pop, q, pop.v0, np.zeros((pop.n, 64)), contact_cap=3)
    _check("free-cubes-cap3", r, y)
    assert ((gst & 2) != 0).sum() >= 5
    balls = P.boxes(32, seed=9, vel_sigma=2.0)
    balls.geom[:, 0] = P.GEOM_SPHERE
    qb = balls.q0.copy()
    qb[:, 2] = rng.uniform(0.03, 0.06, balls.n)
    _check("free-balls", *_one_step(balls, qb, balls.v0, np.zeros((balls.n, 64)))[:2])


def test_free_body_closed_form_matches_the_general_step():
    """The one-body closed form against the general tree step on the same
    cubes: a centre offset of 1e-9 m (negligible, but it makes the engine take
    the general path) gives the same 200-step trajectories within FP32
    rounding."""
    pop = P.boxes(24, seed=13, vel_sigma=2.0).as_float32()
    q = pop.q0.copy()
    q[:, 2] = np.random.default_rng(14).uniform(0.02, 0.3, pop.n)
    Q, V, Sx = S.state_rows(pop, q, pop.v0, np.zeros((pop.n, 64)))
    off = pop.subset(np.arange(pop.n))
    off.com[:, 0, 0] = 1e-9
    out = []
    for p in (pop, off):
        cs = CP.CpuSim()
        cs.set_population(p)
        cs.set_state(Q, V, Sx)
        cs.step(200)
        out.append(cs.read_state())
        cs.close()
    (qa, va, _, sta), (qb, vb, _, stb) = out
    assert np.array_equal(sta, stb) and (sta & 5).sum() == 0
    # measured: 5e-6 m and 8e-6 of the largest velocity component
    assert np.abs(qa[:, :7] - qb[:, :7]).max() < 5e-5
    assert np.abs(va[:, :6] - vb[:, :6]).max() < 1e-4 * max(1.0, np.abs(va[:, :6]).max())


def test_free_body_spin_keeps_the_invariants_of_the_oracle():
    """The one-body closed form on a torque-free box near its intermediate
    axis (no gravity, no ground): world angular momentum and energy drift
    like the oracle's explicit integration (within 2 % and 3 % over 8 s) and
    the spin flips, as it does in the oracle."""
    from tests.test_oracle_pins import _rot_of_quat
    h = np.array([0.05, 0.03, 0.015])
    pop = P.boxes(1, seed=1)
    pop.half[0, 0] = h
    pop = pop.as_float32()
    q = np.array([[0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0]])
    v = np.array([[0.0, 0.0, 0.0, 0.01, 5.0, 0.01]])
    Q, V, Sx = S.state_rows(pop, q, v, np.zeros((1, 64)))
    cs = CP.CpuSim(ground=0, box_box=0, actuate=0, gravity=(0.0, 0.0, 0.0))
    cs.set_population(pop)
    cs.set_state(Q, V, Sx)
    I = np.array([h[1] ** 2 + h[2] ** 2, h[0] ** 2 + h[2] ** 2, h[0] ** 2 + h[1] ** 2]) / 3.0
    L0 = I * v[0, 3:6]
    E0 = 0.5 * np.sum(I * v[0, 3:6] ** 2)
    wy = []
    for _ in range(40):
        cs.step(100)
        qq, vv, _, st = cs.read_state()
        w = vv[0, 3:6].astype(np.float64)
        L = _rot_of_quat(qq[0, 3:7].astype(np.float64)) @ (I * w)
        assert np.linalg.norm(L - L0) <= 0.02 * np.linalg.norm(L0)
        assert abs(0.5 * np.sum(I * w ** 2) - E0) <= 0.03 * E0
        wy.append(w[1])
    cs.close()
    assert st[0] == 0 and min(wy) < -4.5 and max(wy) > 4.5
