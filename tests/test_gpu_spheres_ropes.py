"""Sphere geometry and long chains on the GPU against the FP64 oracle,
through the C ABI.

Scenes: grammar robots whose modules are balls with probability 0.4
(sphere/plane, sphere/box and sphere/sphere contacts), a cube with one ball
(the BOX_AND_BALL-like scene), free balls on an incline (rolling closed form)
and ropes of up to 25 links (the ARM_WITH_ROPE-like long chain).  Bars as in
test_gpu_parity.py (tests/parity.py): 25-link chains, whose mass matrices
reach cond(M) ~ 1e5, are held to the FP32 yardstick like every state where
FP32 arithmetic misses 1e-5, their contact-free flight to twice that
yardstick's drift, and passive ropes, chaotic even in flight, to the
contact-rich bar (population-mean fitness within 2 %).
"""
import numpy as np
import pytest

from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S
from tests.test_cpu_engine import _sphere_contact_kinds, fp32_flight_bar
from tests.test_gpu_parity import MARGIN, _check, _gpu_sim, _one_step, contact_list_matches, ncores, oracle

pytestmark = pytest.mark.gpu


def test_one_step_ball_modules():
    pop = P.grammar(192, seed=81, ball_p=0.4)
    q, v, s = P.random_state(pop, seed=82, angle=1.0)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(83).uniform(-0.05, 0.0, pop.n)
    kinds = _sphere_contact_kinds(pop, q)
    assert kinds.min() >= 10, kinds
    r, y, gst, _ = _one_step(pop, q, v, s)
    _check("ball-modules", r, y)


def test_one_step_box_and_ball():
    pop = P.box_and_ball(128, seed=84)
    q, v, s = P.random_state(pop, seed=85)
    q[:, 2] = np.random.default_rng(86).uniform(0.03, 0.12, pop.n)
    r, y, gst, _ = _one_step(pop, q, v, s)
    _check("box-and-ball", r, y)


def test_sphere_contact_lists_match_oracle():
    """Contact generation with balls, every robot: counts, bodies and order
    exact, geometry to 1e-5 (normals 1e-4), against the oracle's list or one
    of its valid lists where a decision lies near its threshold."""
    O = oracle()
    pop = P.grammar(96, seed=93, ball_p=0.5).as_float32()
    q, v, s = P.random_state(pop, seed=94, angle=1.0)
    q[:, 2] = pop.q0[:, 2] - 0.02
    Q, V, Sx = S.state_rows(pop, q, v, s)
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(1)
    prm = O.default_params()
    with_sphere_pairs = 0
    for i in range(pop.n):
        m = O.model_from_population(pop, i)
        outs, k, complete = O.contact_outcomes(m, Q[i, :O.nq(m)].astype(np.float64), MARGIN, prm)
        g = sm.debug_contacts(i)
        assert contact_list_matches(g, outs, Q[i, :3]), (i, g["n"], [len(c["a"]) for c in outs[:8]], complete)
        c = outs[0]
        with_sphere_pairs += any(b >= 0 and (m.geom[a] or m.geom[b]) for a, b in zip(c["a"], c["b"]))
    assert with_sphere_pairs >= 5, with_sphere_pairs


@pytest.mark.parametrize("alpha_deg,mu,rolls", [(20.0, 0.5, True), (40.0, 0.1, False)])
def test_ball_on_incline_on_gpu(alpha_deg, mu, rolls):
    """Free balls on an incline (tilted gravity): rolling at (5/7) g sin(a)
    with v = omega r when mu >= (2/7) tan(a), else sliding at
    g (sin a - mu cos a); trajectories within 1e-4 m of the oracle."""
    O = oracle()
    G, a, r = 9.81, np.radians(alpha_deg), 0.05
    grav = (G * np.sin(a), 0.0, -G * np.cos(a))
    pop = P.boxes(16, seed=3).as_float32()
    pop.geom[:, 0] = P.GEOM_SPHERE
    pop.half[:, 0] = r
    pop.mass[:, 0] = 0.5
    q = np.zeros((16, 7))
    q[:, 2] = r - 1e-4
    q[:, 3] = 1.0
    q[:, 0] = np.arange(16) * 0.3
    Q, V, Sx = S.state_rows(pop, q, np.zeros((16, 6)), np.zeros((16, 64)))
    sm = _gpu_sim(pop, mu=mu, gravity=grav)
    sm.set_state(Q, V, Sx)
    sm.step(100)
    v0 = sm.read_state()[1].copy()
    sm.step(400)
    gq, gv, _, gst = sm.read_state()
    assert (gst & 5).sum() == 0
    acc = (gv[:, 0] - v0[:, 0]) / (400 * 0.002)
    if rolls:
        assert np.abs(acc - 5.0 / 7.0 * G * np.sin(a)).max() < 0.01 * G * np.sin(a)
        assert np.abs(gv[:, 0] - gv[:, 4] * r).max() < 0.01 * np.abs(gv[:, 0]).min()
    else:
        assert np.abs(acc - G * (np.sin(a) - mu * np.cos(a))).max() < 0.01 * G * np.sin(a)
    oq, _, _, _, _ = O.run_population(pop, Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64), 500,
                                      prm=O.default_params(mu=mu, gravity=grav), threads=ncores())
    assert np.abs(gq[:, :3] - oq[:, :3]).max() <= 1e-4


def test_one_step_ropes_against_the_fp32_yardstick():
    for links in (10, 25):
        pop = P.rope(48, seed=87, links=links)
        q, v, s = P.random_state(pop, seed=88, angle=0.4)
        q[:, 2] = pop.q0[:, 2] + np.random.default_rng(89).uniform(-0.04, 0.0, pop.n)
        r, y, gst, _ = _one_step(pop, q, v, s, actuate=0)
        _check(f"rope-{links}", r, y)


def test_ropes_contact_free_and_contact_rich():
    """Lifted ropes with the servos on, 200 contact-free steps: core within
    1e-4 m of the oracle, or twice the FP32 yardstick's own drift where that
    exceeds 1e-4 m (25 links: cond(M) ~ 1e5 amplifies FP32 rounding step after
    step).  Dropped passive 25-link ropes are chaotic and held to the
    contact-rich bar: population-mean fitness within 2 % after 2000 steps."""
    O = oracle()
    for links in (10, 25):
        pop = P.lift(P.rope(64, seed=91, links=links), 1.0).as_float32()
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        bound, drift = fp32_flight_bar(pop, Q, V, Sx, O.default_params(box_box=0))
        sm = _gpu_sim(pop, box_box=0)
        sm.set_state(Q, V, Sx)
        prm = O.default_params(box_box=0)
        oq, ov, os_ = Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64)
        worst = 0.0
        for _ in range(4):
            sm.step(50)
            oq, ov, os_, _, _ = O.run_population(pop, oq, ov, os_, 50, prm=prm, threads=ncores())
            worst = max(worst, np.abs(sm.read_state()[0][:, :3] - oq[:, :3]).max())
        sm.close()
        print(f"rope-{links} lifted: worst core position error {worst:.3g} m, fp32 yardstick drift {drift:.3g} m")
        assert worst <= bound, (links, worst, drift)
    pop = P.rope(128, seed=92).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    sm = _gpu_sim(pop, actuate=0)
    sm.set_state(Q, V, Sx)
    sm.step(2000)
    gf, st = sm.fitness(), sm.read_state()[3]
    sm.close()
    oq, _, _, ost, _ = O.run_population(pop, pop.q0, pop.v0, P.cpg_initial(pop)[:, :2 * O.MAXB], 2000,
                                        prm=O.default_params(actuate=0), threads=ncores())
    of = O.fitness(pop.q0, oq)
    print("rope mean fitness gpu %.6f oracle %.6f" % (gf.mean(), of.mean()))
    assert (st & 5).sum() == 0 and (ost & 5).sum() == 0
    assert abs(gf.mean() - of.mean()) <= 0.02 * of.mean()


def test_single_free_bodies_on_the_one_body_kernel():
    """Cubes and balls alone take the thread-per-robot kernel: tumbling cubes
    pressed into the ground (with and without a contact cap of 3) and free
    balls against the oracle, one step from the same states."""
    pop = P.boxes(96, seed=7, vel_sigma=2.0)
    rng = np.random.default_rng(8)
    q = pop.q0.copy()
    q[:, 2] = rng.uniform(0.0, 0.09, pop.n)
    for cap in (64, 3):
        r, y, gst, _ = _one_step(pop, q, pop.v0, np.zeros((pop.n, 64)), contact_cap=cap)
        _check(f"free-cubes-cap{cap}", r, y)
        assert np.array_equal(r.status_ref, gst)
    balls = P.boxes(64, seed=9, vel_sigma=2.0)
    balls.geom[:, 0] = P.GEOM_SPHERE
    qb = balls.q0.copy()
    qb[:, 2] = rng.uniform(0.03, 0.06, balls.n)
    r, y, gst, _ = _one_step(balls, qb, balls.v0, np.zeros((balls.n, 64)))
    _check("free-balls", r, y)


def _concat(a, b):
    import dataclasses
    fields = {}
    for f in dataclasses.fields(a):
        x, y = getattr(a, f.name), getattr(b, f.name)
        fields[f.name] = np.concatenate([x, y]) if isinstance(x, np.ndarray) else x
    fields["n"] = a.n + b.n
    return P.Population(**fields)


def test_mixed_population_runs_both_kernels_bitwise():
    """A population mixing free cubes and grammar robots steps each robot
    exactly as a population of its own kind does (the cubes on the
    thread-per-robot kernel, the rest on the warp-per-robot kernel), and the
    contact lists of the cubes match the oracle's."""
    O = oracle()
    cubes = P.boxes(40, seed=11)
    robots = P.grammar(30, seed=12)
    mixed = _concat(robots, cubes).as_float32()
    runs = {}
    for name, pop in (("mixed", mixed), ("robots", robots.as_float32()), ("cubes", cubes.as_float32())):
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        sm = _gpu_sim(pop, warps_per_block=1)
        sm.set_state(Q, V, Sx)
        sm.step(299)
        before = sm.read_state()[0]
        sm.step(1)
        runs[name] = (sm.read_state(), sm, before)
    (qm, vm, sm_, stm), smm, q299 = runs["mixed"]
    assert np.array_equal(qm[:30], runs["robots"][0][0]) and np.array_equal(vm[:30], runs["robots"][0][1])
    assert np.array_equal(qm[30:], runs["cubes"][0][0]) and np.array_equal(vm[30:], runs["cubes"][0][1])
    for i in range(30, 70):
        m = O.model_from_population(mixed, i)
        outs, _, _ = O.contact_outcomes(m, q299[i, :O.nq(m)].astype(np.float64), MARGIN)
        g = smm.debug_contacts(i)
        assert contact_list_matches(g, outs, q299[i, :3]), i
