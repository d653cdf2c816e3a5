"""Long chains: robots of more than 26 bodies (nv > 31), up to 64 bodies
(nv = 69), the rope behind a core of the paper's ARM_WITH_ROPE-like scene.

Oracle pins (CPU, no CUDA): at these sizes the oracle's mass matrix against
the kinetic energy from forward-kinematics differences, its bias forces
against the momentum balance of a free chain, and a ground contact on the
last link against the soft row written with a Jacobian from FK differences.
The host engine refuses chains it does not step.

GPU (through the C ABI, the block-per-robot kernel): one step from random
states against the closest valid outcome of the oracle's step, held to the
FP32 yardstick (tests/parity.py) as every ill-conditioned state is; the
contact lists; contact-free flight against the yardstick's drift; a mixed
population (grammar robots, free cubes, chains) stepping each robot exactly
as a population of its own kind does; graph replay against single launches.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S
from tests import models as H
from tests import parity as PR

G = 9.81


def _rope_model(links, seed=3):
    return O.model_from_population(P.rope(1, seed=seed, links=links), 0)


def _random_state(m, rng, ang=0.5):
    nq, nv = O.nq(m), O.nv(m)
    quat = rng.normal(size=4)
    quat /= np.linalg.norm(quat)
    q = np.concatenate([rng.normal(size=3), quat, rng.uniform(-ang, ang, nq - 7)])
    return q, rng.normal(size=nv)


# ------------------------------------------------------------- oracle pins
def test_long_chain_mass_matrix_against_kinetic_energy():
    """M_ii = 2 T(e_i) and M_ij = T(e_i + e_j) - T(e_i) - T(e_j) with T from
    FK differences (no CRBA code), on a 64-body chain (nv = 69): the diagonal
    and 120 random off-diagonal entries; M symmetric positive definite."""
    m = _rope_model(63)
    assert m.nb == 64 and O.nv(m) == 69
    rng = np.random.default_rng(4)
    q, _ = _random_state(m, rng)
    M = O.mass_matrix(m, q, O.default_params(armature=0.0))
    n = O.nv(m)
    E = np.eye(n)
    T1 = np.array([H.kinetic_energy_fd(m, q, E[i]) for i in range(n)])
    assert np.abs(np.diag(M) - 2 * T1).max() < 1e-6 * np.abs(M).max()
    for _ in range(120):
        i, j = rng.choice(n, 2, replace=False)
        Mij = H.kinetic_energy_fd(m, q, E[i] + E[j]) - T1[i] - T1[j]
        assert abs(M[i, j] - Mij) < 1e-6 * np.abs(M).max(), (i, j)
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0


def test_long_chain_momentum_balance():
    """A free 41-body chain, no contact, no actuation: the rate of linear
    momentum is m_tot g and that of angular momentum about the origin the
    gravity moment, with momenta from FK differences and the acceleration
    M^-1 (-c) of the oracle."""
    m = _rope_model(40)
    rng = np.random.default_rng(9)
    q, v = _random_state(m, rng)
    p = O.default_params(armature=0.0)
    M = O.mass_matrix(m, q, p)
    vdot = np.linalg.solve(M, -O.bias(m, q, v, p))
    qd = H.qdot_from_v(m, q, v)
    h = 1e-4
    Pp, Lp = H.momentum_fd(m, q + h * qd, v + h * vdot)
    Pm, Lm = H.momentum_fd(m, q - h * qd, v - h * vdot)
    dP, dL = (Pp - Pm) / (2 * h), (Lp - Lm) / (2 * h)
    _, _, cc = O.fk(m, q)
    mt = sum(m.mass[b] for b in range(m.nb))
    g = np.array([0.0, 0.0, -G])
    tau_g = sum(np.cross(cc[b], m.mass[b] * g) for b in range(m.nb))
    scale = mt * G * (1 + np.abs(cc).max())
    assert np.abs(dP - mt * g).max() < 2e-5 * scale
    assert np.abs(dL - tau_g).max() < 2e-5 * scale


def _point_velocity_fd(m, q, v, b, p_body, h=1e-7):
    """World velocity of a point fixed in body b, by FK differences."""
    qd = H.qdot_from_v(m, q, v)
    out = []
    for s in (1.0, -1.0):
        R, p, _ = O.fk(m, q + s * h * qd)
        out.append(p[b] + R[b] @ p_body)
    return (out[0] - out[1]) / (2 * h)


def test_tail_contact_obeys_the_soft_row_on_brute_force_jacobian():
    """A straight 40-link chain tilted so that one corner of its last brick
    (body 40) lies 1 mm below the plane, every dof falling at 1 m/s, no
    friction: one contact, whose soft row fixes the corner's normal velocity
    after the step at (R J v_free + A b) / (A + R), with A = J M^-1 J^T,
    R = max(kappa A, min_cfm), b the capped recovery speed (ERP/CFM of the
    stated soft contact).  Here J is the corner's velocity per unit dof
    velocity from FK differences (no Jacobian code of the oracle), and the
    corner's velocity after the step is measured the same way."""
    m = _rope_model(40)
    n = O.nv(m)
    _, p0, _ = O.fk(m, np.concatenate([[0, 0, 0, 1, 0, 0, 0], np.zeros(n - 6)]))
    length = p0[m.nb - 1][0] + 0.06
    Ry = H.rot("y", np.arctan2(0.3, length))       # the tail 0.3 m below the core
    Rx = H.rot("x", 0.05)                           # and one of its sides lower
    Rr = Ry @ Rx
    w = np.sqrt(max(1e-300, 1.0 + np.trace(Rr))) / 2
    quat = np.array([w, (Rr[2, 1] - Rr[1, 2]) / (4 * w), (Rr[0, 2] - Rr[2, 0]) / (4 * w),
                     (Rr[1, 0] - Rr[0, 1]) / (4 * w)])
    q = np.concatenate([[0.0, 0.0, 0.0], quat, np.zeros(n - 6)])
    R, p, _ = O.fk(m, q)
    corners = [np.array([sx * 0.03 + 0.03, sy * 0.03, sz * 0.03]) for sx in (-1, 1) for sy in (-1, 1)
               for sz in (-1, 1)]
    z = {(b, k): (p[b] + R[b] @ c)[2] for b in range(1, m.nb) for k, c in enumerate(corners)}
    (b, k), low = min(z.items(), key=lambda kv: kv[1])
    q[2] = -low - 0.001                            # that corner 1 mm deep, the next one above the plane
    assert sorted(z.values())[1] - low > 0.002
    assert b == m.nb - 1
    v = np.zeros(n)
    v[2] = -1.0
    prm = O.default_params(box_box=0, actuate=0, mu=0.0)
    d = O.step_detail(m, q, v, np.zeros(2 * O.MAXB), prm=prm)
    assert d["nc"] == 1
    c = corners[k]
    J = np.array([_point_velocity_fd(m, q, e, b, c)[2] for e in np.eye(n)])
    assert abs(J[n - 1]) > 0.01 and (np.abs(J[6 + 32:]) > 0.01).sum() >= 4  # hinges past 32 move the corner
    M = O.mass_matrix(m, q, prm)
    A = J @ np.linalg.solve(M, J)
    dt = prm.dt
    om = 2 * np.pi / prm.soft_tau
    kden = dt * om * om + 2 * prm.soft_zeta * om
    erp, kappa = dt * om * om / kden, 1.0 / (dt * kden)
    Rs = max(kappa * A, prm.min_cfm)
    target = min(erp * 0.001 / dt, prm.max_correct_vel)
    pred = (Rs * (J @ d["vfree"]) + A * target) / (A + Rs)
    got = _point_velocity_fd(m, q, d["v"][:n], b, c)[2]
    print(f"tail corner: J v_free {J @ d['vfree']:.4f}, predicted {pred:.6f}, measured {got:.6f} m/s")
    assert abs(got - pred) < 1e-5 * max(1.0, abs(J @ d["vfree"]))
    assert got > J @ d["vfree"] + 0.5                # most of the approach speed removed


def test_host_engine_refuses_long_chains():
    from paper_2502_11129_b300 import cpu as CPU
    pop = P.rope(2, links=30)
    with pytest.raises(Exception, match="bodies"):
        eng = CPU.CpuSim(threads=1)
        eng.set_population(pop)


# ------------------------------------------------------------------- GPU
def _gpu_sim(pop, **cfg):
    sm = S.Sim(**cfg)
    sm.set_population(pop)
    return sm


def _one_step(pop, q, v, s, **cfg):
    pop32 = pop.as_float32()
    Q, V, Sx = S.state_rows(pop32, q, v, s)
    sm = _gpu_sim(pop32, **cfg)
    sm.set_state(Q, V, Sx)
    sm.step(1)
    gq, gv, gs, gst = sm.read_state()
    prm = PR.oracle_params(**cfg)
    r = PR.one_step_errors(pop32, Q, V, Sx, gq, gv, gs, prm)
    y = PR.fp32_yardstick(pop32, Q, V, Sx, prm)
    sm.close()
    return r, y, gst


def _check(name, r, y):
    fails = PR.parity_failures(r, y)
    msg = r.summary(name) + " | fp32 " + y.summary("yardstick") + " | " + "; ".join(fails)
    print(msg)
    assert not fails, msg


@pytest.mark.gpu
@pytest.mark.parametrize("links", [26, 40, 63])
def test_one_step_long_chains(links):
    """Passive chains pushed into the ground from random bent states (contacts
    with the plane and between links, the contact cap reached on the longest),
    one step, every robot against the closest valid oracle outcome."""
    pop = P.rope(24, seed=100 + links, links=links)
    q, v, s = P.random_state(pop, seed=101, angle=0.4)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(102).uniform(-0.04, 0.0, pop.n)
    r, y, gst = _one_step(pop, q, v, s, actuate=0)
    _check(f"chain-{links}", r, y)
    assert np.array_equal(r.status_ref & 2, gst & 2)


@pytest.mark.gpu
def test_one_step_long_chains_actuated():
    """Snakes (the CPG and servos on), 48 links, random states in contact."""
    pop = P.rope(24, seed=110, links=48)
    q, v, s = P.random_state(pop, seed=111, angle=0.6)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(112).uniform(-0.03, 0.0, pop.n)
    r, y, gst = _one_step(pop, q, v, s)
    _check("snake-48", r, y)


def _coiled(links, n, seed, turn=0.3):
    """Chains lying flat, every hinge about the vertical bent by ~turn rad the
    same way: the chain coils, and its tail crosses its head (contacts between
    links far apart in the chain, body indices past 32 included)."""
    pop = P.rope(n, seed=seed, links=links).as_float32()
    m0 = O.model_from_population(pop, 0)
    R, _, _ = O.fk(m0, pop.q0[0, :O.nq(m0)])
    zax = np.round([R[b][:, m0.axis[b]][2] for b in range(1, m0.nb)])
    rng = np.random.default_rng(seed + 1)
    q = pop.q0.copy()
    q[:, 7:7 + links] = turn * zax + rng.uniform(-0.05, 0.05, (n, links))
    q[:, 2] -= 0.01
    v = np.zeros_like(pop.v0)
    v[:, :pop.v0.shape[1]] = rng.normal(0.0, 0.3, pop.v0.shape)
    return pop, q, v, P.cpg_initial(pop)


@pytest.mark.gpu
def test_one_step_coiled_chains():
    """Coiled 40-link snakes: contacts between links and with the plane, the
    contact cap reached, one step against the closest valid oracle outcome."""
    pop, q, v, s = _coiled(40, 24, seed=125)
    r, y, gst = _one_step(pop, q, v, s)
    _check("coiled-40", r, y)


@pytest.mark.gpu
def test_long_chain_contact_lists_match_oracle():
    """Contact generation of coiled 40-link chains, every robot: counts,
    bodies and order exact, geometry to 1e-5, against the oracle's list or
    one of its valid lists where a decision lies near its threshold."""
    from tests.test_gpu_parity import MARGIN, contact_list_matches
    pop, q, v, s = _coiled(40, 24, seed=120)
    Q, V, Sx = S.state_rows(pop, q, v, s)
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(1)
    prm = O.default_params()
    pair_contacts = 0
    for i in range(pop.n):
        m = O.model_from_population(pop, i)
        outs, k, complete = O.contact_outcomes(m, Q[i, :O.nq(m)].astype(np.float64), MARGIN, prm)
        g = sm.debug_contacts(i)
        assert complete, i
        assert contact_list_matches(g, outs, Q[i, :3].astype(np.float64)), (i, g["n"], [len(c["a"]) for c in outs])
        pair_contacts += int(((g["b"] >= 0) & ((g["a"] >= 32) | (g["b"] >= 32))).sum())
    sm.close()
    assert pair_contacts > 10  # body pairs with a body past 32


@pytest.mark.gpu
@pytest.mark.parametrize("actuate", [1, 0])
def test_long_chains_contact_free_flight(actuate):
    """Lifted 40-link chains (snakes and passive ropes), 100 contact-free
    steps: core within 1e-4 m of the oracle, or within twice the FP32
    yardstick's own drift.  (Longer free flights of such chains whip: with
    hinge rates N(0, 1) the tail's rates reach ~100 rad/s by step 100, and
    semi-implicit Euler at dt = 2 ms diverges by step 200 in FP64 as well.)"""
    from tests.test_cpu_engine import fp32_flight_bar
    pop = P.lift(P.rope(32, seed=130, links=40), 1.5).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    prm = O.default_params(box_box=0, actuate=actuate)
    bound, drift = fp32_flight_bar(pop, Q, V, Sx, prm, steps=100)
    sm = _gpu_sim(pop, box_box=0, actuate=actuate)
    sm.set_state(Q, V, Sx)
    sm.step(100)
    gq, _, _, gst = sm.read_state()
    sm.close()
    oq, _, _, ost, _ = O.run_population(pop, Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64),
                                        100, prm=prm, threads=PR.ncores())
    worst = np.abs(gq[:, :3] - oq[:, :3]).max()
    print(f"chain-40 lifted (actuate={actuate}): worst core position error {worst:.3g} m, "
          f"fp32 yardstick drift {drift:.3g} m")
    assert (gst == 0).all() and (ost == 0).all()
    assert worst <= bound


@pytest.mark.gpu
def test_mixed_population_with_chains_bitwise():
    """Grammar robots, free cubes and 40-link chains in one context: every
    robot's state after 300 steps equals that of a population of its own kind
    bit for bit, fitness and status included, and the inspection calls of a
    chain robot return its own contacts and impulses."""
    robots = P.grammar(20, seed=140)
    cubes = P.boxes(10, seed=141)
    chains = P.rope(6, seed=142, links=40)
    mixed = P.concat([chains, robots, cubes]).as_float32()
    out = {}
    for name, pop in (("mixed", mixed), ("chains", chains.as_float32()), ("robots", robots.as_float32()),
                      ("cubes", cubes.as_float32())):
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
        sm = _gpu_sim(pop, warps_per_block=1)
        sm.set_state(Q, V, Sx)
        sm.step(300)
        out[name] = (sm.read_state(), sm.fitness(), sm.debug_contacts(0), sm.debug_solver(0))
        sm.close()
    (qm, vm, smx, stm), fm, cm, dm = out["mixed"]
    for name, sl in (("chains", slice(0, 6)), ("robots", slice(6, 26)), ("cubes", slice(26, 36))):
        (q1, v1, s1, st1), f1, _, _ = out[name]
        assert np.array_equal(qm[sl], q1) and np.array_equal(vm[sl], v1), name
        assert np.array_equal(smx[sl], s1) and np.array_equal(stm[sl], st1), name
        assert np.array_equal(fm[sl], f1), name
    c1, d1 = out["chains"][2], out["chains"][3]
    assert cm["n"] == c1["n"] and np.array_equal(cm["p"], c1["p"])
    assert np.array_equal(dm["vfree"], d1["vfree"]) and np.array_equal(dm["lam"], d1["lam"])
    assert np.abs(qm[:6, 2] - mixed.q0[:6, 2]).max() > 0.01  # the chains did fall


@pytest.mark.gpu
def test_long_chain_graph_replay_equals_single_launches():
    pop = P.rope(8, seed=150, links=45).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    a = _gpu_sim(pop)
    b = _gpu_sim(pop, steps_per_launch=7)
    for sm in (a, b):
        sm.set_state(Q, V, Sx)
    a.step(50)
    for _ in range(5):
        b.step(10)
    qa, va, _, sa = a.read_state()
    qb, vb, _, sb = b.read_state()
    a.close()
    b.close()
    assert np.array_equal(qa, qb) and np.array_equal(va, vb) and np.array_equal(sa, sb)
    assert np.isfinite(qa).all()
