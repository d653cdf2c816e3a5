"""CUDA path vs the FP64 oracle, through the C ABI.

One step from identical FP32-rounded states (tests/parity.py): per robot the
error against the closest valid outcome of the oracle's step (decisions within
1e-5 of their thresholds taken either way), as |dx| / max(|x_ref|, 1) for each
of q, v and the CPG state (the stated 1e-5 bar) and as the worst single entry;
every robot is compared.  Where FP32 arithmetic itself meets 1e-5 on every
robot of the states (the oracle's FP32 build on the same states), the GPU must
too; on ill-conditioned states (settled, servo-loaded robots) the GPU's error
distribution may be no worse than that FP32 yardstick's.  Contact-free robots
(lifted 1 m): core position within 1e-4 m over 200 steps.  Contact-rich runs
(chaotic): population-mean fitness within 2 %.
"""
import numpy as np
import pytest

from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S
from tests import parity as PR

pytestmark = pytest.mark.gpu

MARGIN = PR.BAND
ncores = PR.ncores


def oracle():
    from oracle import oracle as O
    return O


def _gpu_sim(pop, **cfg):
    sm = S.Sim(**cfg)
    sm.set_population(pop)
    return sm


def _one_step(pop, q, v, s, **cfg):
    """One GPU step from the FP32-rounded states; returns (errors against the
    oracle's closest valid outcome, FP32 yardstick errors, GPU status bits,
    the simulator)."""
    pop32 = pop.as_float32()
    Q, V, Sx = S.state_rows(pop32, q, v, s)
    sm = _gpu_sim(pop32, **cfg)
    sm.set_state(Q, V, Sx)
    sm.step(1)
    gq, gv, gs, gst = sm.read_state()
    prm = PR.oracle_params(**cfg)
    r = PR.one_step_errors(pop32, Q, V, Sx, gq, gv, gs, prm)
    y = PR.fp32_yardstick(pop32, Q, V, Sx, prm)
    return r, y, gst, sm


def _check(name, r, y):
    fails = PR.parity_failures(r, y)
    msg = r.summary(name) + " | fp32 " + y.summary("yardstick") + " | " + "; ".join(fails)
    print(msg)
    assert not fails, msg


def test_one_step_free_boxes():
    pop = P.boxes(64, seed=1)
    q = pop.q0.copy()
    q[:32, 2] = np.random.default_rng(0).uniform(0.03, 0.08, 32)  # half of them in contact
    r, y, gst, _ = _one_step(pop, q, pop.v0, np.zeros((64, 64)))
    _check("boxes", r, y)
    assert np.array_equal(r.status_ref, gst)


def test_one_step_quadrupeds_random_states():
    pop = P.quadrupeds(128, seed=2)
    q, v, s = P.random_state(pop, seed=5)
    q[:, 2] = np.random.default_rng(1).uniform(0.03, 0.09, pop.n)
    r, y, gst, _ = _one_step(pop, q, v, s)
    _check("quadrupeds", r, y)


def test_one_step_grammar_random_states():
    pop = P.grammar(256, seed=3)
    q, v, s = P.random_state(pop, seed=7)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(2).uniform(-0.04, 0.0, pop.n)
    r, y, gst, _ = _one_step(pop, q, v, s)
    _check("grammar", r, y)


def test_one_step_grammar_zero_pose_settled_by_oracle():
    """States taken from an oracle run (realistic contact sets) at step 300:
    resting, servo-loaded robots whose mass matrices reach cond ~ 2e4, where
    FP32 arithmetic alone does not hold 1e-5 on every robot."""
    O = oracle()
    pop = P.grammar(96, seed=13).as_float32()
    q, v, s, st, _ = O.run_population(pop, pop.q0, pop.v0, P.cpg_initial(pop), 300, threads=ncores())
    r, y, gst, _ = _one_step(pop, q, v, s)
    _check("grammar-settled", r, y)


def contact_list_matches(g, outs, origin):
    """The GPU's contact list equals one of the valid oracle lists: counts,
    bodies and order exactly, depths and points to 1e-5, normals to 1e-4."""
    for c in outs:
        if (g["n"] == len(c["a"]) and np.array_equal(g["a"], c["a"]) and np.array_equal(g["b"], c["b"])
                and np.allclose(g["depth"], c["depth"], atol=1e-5) and np.allclose(g["nrm"], c["n"], atol=1e-4)
                and np.allclose(g["p"], c["p"] - origin, atol=1e-5)):
            return True
    return False


def test_contact_lists_match_oracle():
    """Contact generation, every robot: counts, bodies and order exact,
    geometry to 1e-5, against the oracle's list or, where a decision lies
    within 1e-5 of its threshold, one of its valid lists."""
    O = oracle()
    pop = P.grammar(64, seed=31).as_float32()
    q, v, s = P.random_state(pop, seed=9, angle=1.0)
    q[:, 2] = pop.q0[:, 2] - 0.02
    Q, V, Sx = S.state_rows(pop, q, v, s)
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(1)
    prm = O.default_params()
    near = 0
    for i in range(pop.n):
        m = O.model_from_population(pop, i)
        outs, k, complete = O.contact_outcomes(m, Q[i, :O.nq(m)].astype(np.float64), MARGIN, prm)
        near += k > 0
        g = sm.debug_contacts(i)
        assert contact_list_matches(g, outs, Q[i, :3]), (i, g["n"], [len(c["a"]) for c in outs[:8]], complete)
    print("contact lists: robots with near-threshold decisions", near, "of", pop.n)


def test_contact_free_trajectories_200_steps():
    """Lifted 1 m, no box/box: core position within 1e-4 m of the oracle
    for 200 steps (0.4 s of fall, no ground contact yet)."""
    O = oracle()
    for pop in (P.quadrupeds(64, seed=2), P.grammar(128, seed=3)):
        pop = P.lift(pop, 1.0).as_float32()
        s0 = P.cpg_initial(pop)
        Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
        sm = _gpu_sim(pop, box_box=0)
        sm.set_state(Q, V, Sx)
        prm = O.default_params(box_box=0)
        oq, ov, os_ = Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64)
        worst = 0.0
        for chunk in range(4):
            sm.step(50)
            gq, _, _, _ = sm.read_state()
            oq, ov, os_, st, _ = O.run_population(pop, oq, ov, os_, 50, prm=prm, threads=ncores())
            worst = max(worst, np.abs(gq[:, :3] - oq[:, :3]).max())
        print(pop.kind, "worst core position error", worst)
        assert worst <= 1e-4


def test_population_mean_fitness_contact_rich():
    """1024 quadrupeds x 5000 steps: chaos forbids trajectory matching; the
    population-mean fitness must agree within 2 %."""
    O = oracle()
    pop = P.quadrupeds(1024, seed=2).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(5000)
    gf = sm.fitness()
    _, _, _, gst = sm.read_state()
    oq, _, _, ost, _ = O.run_population(pop, pop.q0, pop.v0, s0[:, :2 * O.MAXB], 5000, threads=ncores())
    of = O.fitness(pop.q0, oq)
    print("mean fitness gpu %.6f oracle %.6f" % (gf.mean(), of.mean()))
    assert (gst & 5).sum() == 0 and (ost & 5).sum() == 0
    assert abs(gf.mean() - of.mean()) <= 0.02 * of.mean()


def test_status_nonfinite_freezes_only_that_variant():
    pop = P.quadrupeds(8, seed=2).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    V[3, 7] = np.nan
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(20)
    gq, gv, gs, st = sm.read_state()
    assert st[3] & S.ST_NONFINITE
    assert np.array_equal(gq[3], Q[3])
    others = np.delete(np.arange(8), 3)
    assert np.all(st[others] & 5 == 0)
    assert np.all(np.isfinite(gq[others]))
    assert np.abs(gq[others, :3] - Q[others, :3]).max() > 0  # they moved


def test_abi_errors_on_device():
    sm = S.Sim()
    with pytest.raises(S.SimError, match="SIM_ESTATE"):
        sm.step(1)
    pop = P.quadrupeds(2)
    bad = pop.subset([0, 1])
    bad.parent[1, 3] = 5  # parent must precede the child
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        sm.set_population(bad)
    sm.set_population(pop)
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        sm.read_state(first=1, count=5)
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        sm.step(-1)
    sm.close()


def test_graph_replay_matches_single_launches():
    """A step count captured as a graph of chunked persistent launches gives
    the same state as steps issued one by one (bitwise: same kernels)."""
    pop = P.grammar(64, seed=41).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    a = _gpu_sim(pop, steps_per_launch=7)
    a.set_state(Q, V, Sx)
    a.step(40)
    b = _gpu_sim(pop, steps_per_launch=40)
    b.set_state(Q, V, Sx)
    b.step(40)
    qa, va, _, _ = a.read_state()
    qb, vb, _, _ = b.read_state()
    assert np.array_equal(qa, qb) and np.array_equal(va, vb)


def test_autotune_keeps_state():
    pop = P.grammar(200, seed=43).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    a = _gpu_sim(pop)
    a.set_state(Q, V, Sx)
    a.autotune(20)
    q1, v1, _, _ = a.read_state()
    assert np.array_equal(q1, Q) and np.array_equal(v1, V)
    shape = a.launch_shape()
    assert shape["warps_per_sm"] in (12, 16) and shape["warps_per_block"] in (1, 2, 4, 8)
    assert not (shape["warps_per_sm"] == 12 and shape["warps_per_block"] == 8)
    a.step(30)
    b = _gpu_sim(pop, warps_per_block=1)
    b.set_state(Q, V, Sx)
    b.step(30)
    assert np.array_equal(a.read_state()[0], b.read_state()[0])
    # a configured register budget is kept by the autotuner
    c = _gpu_sim(pop, warps_per_sm=12)
    c.set_state(Q, V, Sx)
    c.autotune(20)
    assert c.launch_shape()["warps_per_sm"] == 12
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        S.Sim(warps_per_sm=12, warps_per_block=8)
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        S.Sim(warps_per_sm=10)


def test_launch_shapes_and_phase_lock_agree_bitwise():
    """Warps per block, phase-locked blocks (with idle warps in the last
    block and a frozen robot that keeps taking the barriers), the register
    budget (16 or 12 resident warps per SM) and the slowest-first launch
    order change only the schedule: every robot's state is bitwise the
    same."""
    pop = P.grammar(203, seed=47).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    V[5, 8] = np.nan  # robot 5 freezes at its first step
    ref = None
    for wpb, lock, occ in ((1, 0, 16), (2, 1, 16), (4, 0, 16), (4, 1, 16), (8, 1, 16), (1, 0, 12), (2, 1, 12),
                           (4, 0, 12)):
        sm = _gpu_sim(pop, warps_per_block=wpb, phase_lock=lock, warps_per_sm=occ, steps_per_launch=25)
        sm.set_state(Q, V, Sx)
        sm.step(60)
        out = sm.read_state()
        sm.close()
        assert out[3][5] & S.ST_NONFINITE and np.array_equal(out[0][5], Q[5])
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b, equal_nan=True), (wpb, lock, occ)


def test_one_step_largest_robots_26_bodies():
    """The largest robots of the warp-per-robot kernel (25 hinges: 26 bodies,
    31 dofs, every lane of the warp a dof) in random poses against the oracle."""
    pop = P.grammar(48, seed=51, hinges=(25, 25))
    assert (pop.nb == S.SIM_WARP_MAX_BODIES).all()
    q, v, s = P.random_state(pop, seed=52)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(53).uniform(-0.03, 0.0, pop.n)
    r, y, gst, _ = _one_step(pop, q, v, s)
    # lattice-aligned bricks in random poses sit in exact separating-axis
    # ties: those robots are compared with the closest valid outcome
    _check("grammar-26-bodies", r, y)


def _contact_counts(sm, n):
    return np.array([sm.debug_solver(i)["n"] for i in range(n)])


def test_one_step_both_sweep_paths_and_the_contact_cap():
    """Robots pushed into the ground so that steps have at most 10 contacts
    (lane-per-row sweep) as well as more (lane-per-contact sweep), then the same
    states with a cap of 6 (overflow: the 6 deepest kept in list order) --
    each against the oracle."""
    pop = P.grammar(128, seed=61)
    q, v, s = P.random_state(pop, seed=62, angle=0.3)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(63).uniform(-0.06, -0.005, pop.n)
    r, y, gst, sm = _one_step(pop, q, v, s)
    nc = _contact_counts(sm, pop.n)
    print("contact counts", np.bincount(nc))
    assert (nc <= 10).sum() >= 10 and (nc > 10).sum() >= 10, np.bincount(nc)
    _check("both-sweeps", r, y)
    r, y, gst, sm = _one_step(pop, q, v, s, contact_cap=6)
    nc = _contact_counts(sm, pop.n)
    over = (gst & S.ST_OVERFLOW) != 0
    assert over.sum() >= 20 and (nc <= 6).all()
    assert np.array_equal(over, (r.status_ref & S.ST_OVERFLOW) != 0)
    _check("cap-6", r, y)


def test_one_step_three_sweep_paths():
    """Large robots pushed deep into the ground so that the three formulations
    of the sweep all run in one launch: at most 10 contacts (contact space,
    lane = row), 11 to 32 (contact space, lane = contact, Delassus blocks in
    the scratch) and more (dof space) -- every robot against the oracle."""
    pop = P.grammar(48, seed=71, hinges=(20, 25))
    q, v, s = P.random_state(pop, seed=72, angle=0.3)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(73).uniform(-0.08, -0.03, pop.n)
    r, y, gst, sm = _one_step(pop, q, v, s)
    nc = _contact_counts(sm, pop.n)
    print("contact counts", np.bincount(nc))
    assert (nc <= 10).sum() >= 5 and ((nc > 10) & (nc <= 32)).sum() >= 5 and (nc > 32).sum() >= 5, nc
    _check("three-sweeps", r, y)


def test_empty_and_ragged_inputs():
    """n = 0 is rejected, a zero-count state transfer is a no-op, and a
    population whose size is no multiple of any launch shape steps every
    robot exactly (ragged last block) -- checked against one-robot runs."""
    sm = S.Sim()
    empty = P.grammar(3, seed=71).subset(np.zeros(0, np.int64))
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        sm.set_population(empty)
    pop = P.grammar(37, seed=72).as_float32()
    sm.set_population(pop)
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    sm.set_state(Q[:0], V[:0], Sx[:0])
    sm.set_state(Q, V, Sx)
    sm.step(25)
    gq = sm.read_state()[0]
    sm.close()
    for i in (0, 17, 36):
        one = _gpu_sim(pop.subset([i]))
        one.set_state(Q[i:i + 1], V[i:i + 1], Sx[i:i + 1])
        one.step(25)
        assert np.array_equal(one.read_state()[0][0], gq[i])
        one.close()


def test_bench_workload_full_size_sampled_one_step():
    """The timed workload at full size (4096 grammar robots, seed 3) in the
    bench's launch configuration (autotuned shape, 500-step launches, CUDA
    graph, slowest-first order): after 1000 steps, one more step of every
    16th robot from the GPU's FP32 state against the oracle from the same
    state (the bars of tests/parity.py: settled robots, the FP32
    yardstick)."""
    O = oracle()
    pop = P.grammar(4096, seed=3).as_float32()
    s0 = P.cpg_initial(pop)
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, s0)
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.autotune(100)
    sm.set_state(Q, V, Sx)
    sm.step(1000)
    Q1, V1, S1, st1 = sm.read_state()
    sm.close()
    idx = np.arange(0, 4096, 16)
    idx = idx[(st1[idx] & 5) == 0]
    sub = pop.subset(idx)
    r, y, gst, _ = _one_step(sub, Q1[idx].astype(np.float64), V1[idx].astype(np.float64),
                             S1[idx].astype(np.float64))
    _check("bench-4096-sampled", r, y)


@pytest.mark.parametrize("alpha_deg,slides", [(20.0, False), (35.0, True)])
def test_incline_stick_slide_on_gpu(alpha_deg, slides):
    """Tilted gravity on a flat plane = an incline (mu = 0.5, tan a vs mu):
    free cubes resting on it stick below the friction angle and slide with
    deceleration g (sin a - mu cos a) above it; the trajectory matches the
    oracle within 1e-4 m over 500 steps."""
    O = oracle()
    G = 9.81
    a = np.radians(alpha_deg)
    grav = (G * np.sin(a), 0.0, -G * np.cos(a))
    pop = P.boxes(16, seed=3).as_float32()
    q = np.zeros((16, 7))
    q[:, 2] = 0.0499
    q[:, 3] = 1.0
    q[:, 0] = np.arange(16) * 0.3  # the robots are independent anyway
    v = np.zeros((16, 6))
    Q, V, Sx = S.state_rows(pop, q, v, np.zeros((16, 64)))
    sm = _gpu_sim(pop, mu=0.5, gravity=grav)
    sm.set_state(Q, V, Sx)
    sm.step(100)
    v_before = sm.read_state()[1][:, 0].copy()
    sm.step(400)
    gq, gv, _, gst = sm.read_state()
    assert (gst & 5).sum() == 0
    if slides:
        acc = (gv[:, 0] - v_before) / (400 * 0.002)
        assert np.abs(acc - G * (np.sin(a) - 0.5 * np.cos(a))).max() < 0.01 * G * np.sin(a)
    else:
        assert np.abs(gv[:, 0]).max() < 0.02
        assert np.abs(gq[:, 0] - q[:, 0]).max() < 0.02
    prm = O.default_params(mu=0.5, gravity=grav)
    oq, _, _, _, _ = O.run_population(pop, Q.astype(np.float64), V.astype(np.float64), Sx.astype(np.float64), 500,
                                      prm=prm, threads=ncores())
    assert np.abs(gq[:, :3] - oq[:, :3]).max() <= 1e-4


def test_heavy_cubes_rest_on_the_softness_floor_on_gpu():
    """100 kg cubes (kappa A below min_cfm): the GPU's steady depth equals the
    closed form min_cfm lambda dt / ERP within 1e-6 m."""
    pop = P.boxes(8, seed=5).as_float32()
    pop.mass[:, 0] = 100.0
    q = np.zeros((8, 7))
    q[:, 2] = 0.0501
    q[:, 3] = 1.0
    Q, V, Sx = S.state_rows(pop, q, np.zeros((8, 6)), np.zeros((8, 64)))
    sm = _gpu_sim(pop)
    sm.set_state(Q, V, Sx)
    sm.step(4000)
    gq, gv, _, gst = sm.read_state()
    dt, G = 0.002, 9.81
    omg = 2 * np.pi / 0.02
    kden = dt * omg * omg + 2 * omg
    erp = dt * omg * omg / kden
    dstar = 0.1 * (100.0 * G * dt / 4) * dt / erp
    assert (gst & 5).sum() == 0
    assert np.abs(gq[:, 2] - (0.05 - dstar)).max() < 1e-6


def test_device_buffer_state_transfers_match_host_ones():
    """sim_set_state_dev / sim_read_state_dev / sim_fitness_dev with CUDA
    torch tensors give bitwise the results of the host-buffer calls, and a
    host pointer is refused."""
    import torch
    pop = P.grammar(77, seed=91).as_float32()
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    a = _gpu_sim(pop)
    a.set_state(Q, V, Sx)
    a.step(40)
    qa, va, sa, sta = a.read_state()
    fa = a.fitness()
    b = _gpu_sim(pop)
    dev = torch.device("cuda", 0)
    tq, tv, ts = (torch.from_numpy(x).to(dev) for x in (Q, V, Sx))
    torch.cuda.synchronize()
    b.set_state_dev(0, pop.n, tq.data_ptr(), tv.data_ptr(), ts.data_ptr())
    b.step(40)
    oq = torch.zeros_like(tq)
    ov = torch.zeros_like(tv)
    os_ = torch.zeros_like(ts)
    ost = torch.zeros(pop.n, dtype=torch.int32, device=dev)
    of = torch.zeros(pop.n, dtype=torch.float32, device=dev)
    b.read_state_dev(0, pop.n, oq.data_ptr(), ov.data_ptr(), os_.data_ptr(), ost.data_ptr())
    b.fitness_dev(of.data_ptr())
    ext = torch.cuda.ExternalStream(b.stream, device=dev)
    ext.synchronize()
    assert np.array_equal(oq.cpu().numpy(), qa) and np.array_equal(ov.cpu().numpy(), va)
    assert np.array_equal(os_.cpu().numpy(), sa)
    assert np.array_equal(ost.cpu().numpy().view(np.uint32), sta)
    assert np.array_equal(of.cpu().numpy(), fa)
    # a part of the population, and a host buffer refused
    b.read_state_dev(10, 5, q_ptr=oq.data_ptr())
    ext.synchronize()
    assert np.array_equal(oq[:5].cpu().numpy(), qa[10:15])
    with pytest.raises(S.SimError, match="SIM_EINVAL"):
        b.set_state_dev(0, 2, Q.ctypes.data, V.ctypes.data)
