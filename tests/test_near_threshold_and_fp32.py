"""The two instruments the parity bars rest on (CPU only).

* Valid outcomes of a step (oracle.step_outcomes): with no decision reversed
  the step is exactly the oracle's; a decision within the band of its
  threshold, reversed, gives the other branch (a contact dropped or added,
  the runner-up axis); decisions outside the band are never reversed.
* The FP32 yardstick (oracle32: the oracle's source evaluated in FP32): on
  random states it meets the stated 1e-5 per-step bar on every robot, on
  settled, servo-loaded robots it does not (the premise of the two-regime bar
  in tests/parity.py), and the host engine, a second FP32 implementation,
  matches its error distribution there.
"""
import numpy as np

from oracle import oracle as O
from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S
from tests import models as H
from tests import parity as PR


def _cube(z, tilt=0.0):
    m = H.single_box(0.05, 1.0)
    q = np.array([0.0, 0.0, z, np.cos(tilt / 2), np.sin(tilt / 2), 0.0, 0.0])
    return m, q


def test_no_reversal_is_the_plain_step_bitwise():
    pop = P.grammar(12, seed=21).as_float32()
    q, v, s = P.random_state(pop, seed=22)
    q[:, 2] = pop.q0[:, 2] - 0.01
    for i in range(pop.n):
        m = O.model_from_population(pop, i)
        nq, nv = O.nq(m), O.nv(m)
        s64 = np.zeros(2 * O.MAXB)
        s64[:2 * (m.nb - 1)] = s[i, :2 * (m.nb - 1)]
        a = O.run(m, q[i, :nq], v[i, :nv], s64, 1)
        b = O.step_flip(m, q[i, :nq], v[i, :nv], s64, (), band=1e-5)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        assert a[3] == b[3]


def test_a_vertex_at_the_plane_is_a_two_way_decision():
    """A cube tilted about x so that one edge's two vertices sit 2e-7 m below
    the plane and the rest well above: the plain step has those two vertex
    contacts; reversing each near decision drops one of them; the tree has
    the four combinations."""
    h = 0.05
    m, q = _cube(0.0)
    # rotate 30 deg about x, then lift so the lowest edge is 2e-7 m deep
    t = np.radians(30.0)
    q[3:7] = [np.cos(t / 2), np.sin(t / 2), 0.0, 0.0]
    low = h * (np.cos(t) + np.sin(t))
    q[2] = low - 2e-7
    c = O.contacts(m, q, O.default_params())
    assert len(c["a"]) == 2 and np.allclose(c["depth"], 2e-7, atol=1e-12)
    cl, k, complete = O.contact_outcomes(m, q, band=1e-5)
    assert k == 2 and complete
    counts = sorted(len(x["a"]) for x in cl)
    assert counts == [0, 1, 1, 2]
    # outside the band nothing is reversed
    cl, k, _ = O.contact_outcomes(m, q, band=1e-8)
    assert k == 0 and len(cl) == 1


def test_runner_up_axis_on_an_exact_separating_axis_tie():
    """A small cube resting 1 mm into a larger one: the two boxes' z faces
    overlap by exactly the same 1 mm (an exact tie, taken by the lower axis:
    the larger box's face is the reference).  Reversing the tie makes the
    small box's face the reference; both outcomes are the same four-point
    patch of depth 1 mm with the normal from the upper box to the lower, on
    one or the other surface."""
    d = 0.001
    bodies = [dict(half=(0.05, 0.05, 0.05), mass=1.0),
              dict(parent=0, axis=1, p_fix=(0.0, 1.0, 0.0), half=(0.03, 0.03, 0.03)),
              dict(parent=0, axis=1, p_fix=(0.004, 1.003, 0.05 - d), half=(0.02, 0.02, 0.02))]
    m = H.make_model(bodies, root_fixed=True, root_p=(0.0, 0.0, 5.0))
    cl, k, complete = O.contact_outcomes(m, np.zeros(2), band=1e-5, prm=O.default_params(ground=0))
    assert complete and k >= 1 and len(cl) >= 2
    zs = set()
    for x in cl:
        if len(x["a"]) != 4:
            continue
        assert np.allclose(x["depth"], d, atol=1e-12)
        assert np.allclose(x["n"], [[0.0, 0.0, -1.0]] * 4, atol=1e-12)
        zs.add(round(float(x["p"][0, 2] - 5.0), 9))
    assert zs == {round(0.03 - d, 9), 0.03}, zs  # the small box's bottom face or the large box's top face


def _settled(n=48, seed=13, steps=300):
    pop = P.grammar(n, seed=seed).as_float32()
    q, v, s, _, _ = O.run_population(pop, pop.q0, pop.v0, P.cpg_initial(pop), steps, threads=PR.ncores())
    return pop, S.state_rows(pop, q, v, s)


def test_fp32_arithmetic_meets_1e5_on_random_states_but_not_on_settled_robots():
    pop = P.grammar(96, seed=3).as_float32()
    q, v, s = P.random_state(pop, seed=7)
    q[:, 2] = pop.q0[:, 2] + np.random.default_rng(2).uniform(-0.04, 0.0, pop.n)
    Q, V, Sx = S.state_rows(pop, q, v, s)
    y = PR.fp32_yardstick(pop, Q, V, Sx)
    print(y.summary("random fp32"))
    assert (y.e_norm <= PR.TOL_STEP).all()
    pop, (Q, V, Sx) = _settled()
    y = PR.fp32_yardstick(pop, Q, V, Sx)
    print(y.summary("settled fp32"))
    assert (y.e_norm > PR.TOL_STEP).any()       # 1e-5 per robot is beyond FP32 here
    assert np.median(y.e_norm) < PR.TOL_STEP    # ... but not by much
    assert y.e_norm.max() < PR.CAP_NORM


def test_fp32_yardstick_is_the_same_code_evaluated_in_fp32():
    """On a free fall (no contact) the FP32 build follows the exact discrete
    closed form to FP32 rounding, like the FP64 build to FP64 rounding."""
    from oracle import oracle32 as O32
    pop = P.boxes(4, seed=1).as_float32()
    q = pop.q0.copy()
    q[:, 2] = 2.0
    v = np.zeros((4, 6))
    v[:, 2] = 1.0
    Q, V, Sx = S.state_rows(pop, q, v, np.zeros((4, 64)))
    n, dt, g = 100, 0.002, 9.81
    z = 2.0 + n * dt * 1.0 - g * dt * dt * n * (n + 1) / 2
    fq = O32.run_population(pop, Q, V, Sx, n, prm=O.default_params(ground=0))[0]
    oq = O.run_population(pop, Q.astype(float), V.astype(float), Sx.astype(float), n,
                          prm=O.default_params(ground=0))[0]
    assert np.abs(oq[:, 2] - z).max() < 1e-12
    assert 1e-9 < np.abs(fq[:, 2] - z).max() < 1e-5
