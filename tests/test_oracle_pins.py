"""Pins of the FP64 oracle against closed forms, brute force and invariants.

These tests never use the CUDA path.  Each pin checks the oracle against
something other than itself: a textbook closed form, a brute-force quantity
computed from forward-kinematics finite differences, or an exact invariant of
the mathematics.  A plausible mistake (dropped term, wrong sign or index,
transposed operand) in the oracle fails at least one of them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2502_11129_b300 import population as P
from tests import models as H

G = 9.81


def prm(**kw):
    base = dict(ground=0, box_box=0, actuate=0)
    base.update(kw)
    return O.default_params(**base)


def free_q(p=(0.0, 0.0, 1.0), quat=(1.0, 0.0, 0.0, 0.0), hinges=()):
    return np.array(list(p) + list(quat) + list(hinges), dtype=float)


# ------------------------------------------------------------ integration
def test_free_fall_exact_discrete_closed_form():
    """Semi-implicit Euler under gravity: z_n = z0 + n dt vz - g dt^2 n(n+1)/2."""
    m = H.single_box()
    dt, n = 0.002, 400
    q0 = free_q((0.3, -0.2, 10.0))
    v0 = np.array([0.7, -0.4, 1.5, 0, 0, 0], float)
    q, v, _, st, _ = O.run(m, q0, v0, np.zeros(2), n, prm=prm(dt=dt))
    assert st == 0
    z = q0[2] + n * dt * v0[2] - G * dt * dt * n * (n + 1) / 2
    assert abs(q[2] - z) < 1e-12
    # projectile: horizontal motion is linear in time
    assert abs(q[0] - (q0[0] + n * dt * v0[0])) < 1e-12
    assert abs(q[1] - (q0[1] + n * dt * v0[1])) < 1e-12
    assert abs(v[2] - (v0[2] - G * dt * n)) < 1e-11


def test_isotropic_cube_torque_free_rotation_is_exact():
    """A cube has isotropic inertia: omega x I omega = 0, so the body rate and
    the world angular momentum R I omega stay constant (the exponential map
    rotates about omega itself)."""
    m = H.single_box()
    w0 = np.array([1.0, 2.0, -0.5])
    q0 = free_q((0, 0, 1), quat=np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2]))
    v0 = np.concatenate([[0.0, 0.0, 0.0], w0])
    q, v, _, st, _ = O.run(m, q0, v0, np.zeros(2), 1000, prm=prm(gravity=(0, 0, 0)))
    assert np.allclose(v[3:6], w0, atol=1e-12)
    R0, _, _ = O.fk(m, q0)
    R1, _, _ = O.fk(m, q)
    I = H.box_inertia_body(m, 0)
    L0 = R0[0] @ (I * w0)
    L1 = R1[0] @ (I * v[3:6])
    assert np.linalg.norm(L1 - L0) < 1e-12 * np.linalg.norm(L0) * 1000
    # the rotation did happen: 1000 steps at |w| = 2.29 rad/s over 2 s
    assert np.linalg.norm(R1[0] - R0[0]) > 0.5


# ---------------------------------------------------------------------- FK
def test_fk_hand_computed_quadruped_leg():
    """Hip on the +x face (hinge vertical), knee on the hip's outer face.

    Hip joint frame Rx(90 deg): its hinge (child y) is world z.  With the hip
    turned by 90 deg the leg points along +y.  Worked by hand:
      R_hip   = [[0,0,1],[1,0,0],[0,1,0]],   hip centre  = p0 + (0.05, 0.03, 0)
      R_knee  = [[0,1,0],[1,0,0],[0,0,-1]],  knee origin = p0 + (0.05, 0.06, 0)
      knee centre = p0 + (0.05, 0.09, 0).
    """
    pop = P.quadrupeds(1)
    m = O.model_from_population(pop, 0)
    p0 = np.array([1.0, 2.0, 3.0])
    hinges = np.zeros(8)
    hinges[0] = np.pi / 2          # body 1 = hip on +x
    q = free_q(p0, hinges=hinges)
    R, p, c = O.fk(m, q)
    assert np.allclose(R[1], [[0, 0, 1], [1, 0, 0], [0, 1, 0]], atol=1e-15)
    assert np.allclose(c[1], p0 + [0.05, 0.03, 0.0], atol=1e-15)
    assert np.allclose(R[5], [[0, 1, 0], [1, 0, 0], [0, 0, -1]], atol=1e-15)
    assert np.allclose(p[5], p0 + [0.05, 0.06, 0.0], atol=1e-15)
    assert np.allclose(c[5], p0 + [0.05, 0.09, 0.0], atol=1e-15)
    # whole robot yawed by +90 deg through the root quaternion, hinges at 0:
    # the +x hip moves to +y, its centre at p0 + (0, 0.08, 0)
    q = free_q(p0, quat=(np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)), hinges=np.zeros(8))
    R, p, c = O.fk(m, q)
    assert np.allclose(c[1], p0 + [0.0, 0.08, 0.0], atol=1e-15)
    assert np.allclose(c[5], p0 + [0.0, 0.14, 0.0], atol=1e-15)


# -------------------------------------------------------------------- CRBA
def _random_state(m, rng, ang=0.8):
    nq, nv = O.nq(m), O.nv(m)
    if m.root_fixed:
        q = rng.uniform(-ang, ang, nq)
    else:
        quat = rng.normal(size=4)
        quat /= np.linalg.norm(quat)
        q = np.concatenate([rng.normal(size=3), quat, rng.uniform(-ang, ang, nq - 7)])
    v = rng.normal(size=nv)
    return q, v


def _small_models():
    out = []
    g = P.grammar(12, seed=11, hinges=(2, 3))
    for i in range(g.n):
        out.append(O.model_from_population(g, i))
    out.append(O.model_from_population(P.quadrupeds(1), 0))
    return out


def test_mass_matrix_matches_kinetic_energy_brute_force():
    """M_ij = T(e_i + e_j) - T(e_i) - T(e_j), with the kinetic energy T built
    from finite differences of FK positions and rotations (no CRBA code)."""
    rng = np.random.default_rng(5)
    for m in _small_models():
        q, _ = _random_state(m, rng)
        M = O.mass_matrix(m, q, O.default_params(armature=0.0))
        n = O.nv(m)
        E = np.eye(n)
        T1 = [H.kinetic_energy_fd(m, q, E[i]) for i in range(n)]
        Mb = np.zeros((n, n))
        for i in range(n):
            Mb[i, i] = 2 * T1[i]
            for j in range(i + 1, n):
                Mb[i, j] = Mb[j, i] = H.kinetic_energy_fd(m, q, E[i] + E[j]) - T1[i] - T1[j]
        assert np.abs(M - Mb).max() < 1e-6 * np.abs(Mb).max()
        assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
        assert np.linalg.eigvalsh(M).min() > 0


def test_mass_matrix_armature_on_hinge_diagonal_only():
    m = O.model_from_population(P.quadrupeds(1), 0)
    q, _ = _random_state(m, np.random.default_rng(1))
    M0 = O.mass_matrix(m, q, O.default_params(armature=0.0))
    M1 = O.mass_matrix(m, q, O.default_params(armature=0.25))
    D = M1 - M0
    assert np.allclose(np.diag(D)[6:], 0.25, atol=1e-15)
    assert np.allclose(np.diag(D)[:6], 0.0, atol=1e-15)
    assert np.abs(D - np.diag(np.diag(D))).max() == 0.0


# -------------------------------------------------------------------- RNEA
def _fixed_root(m, rng):
    m.root_fixed = 1
    Rr = H.rot("z", 0.3) @ H.rot("x", 0.2)
    for k in range(9):
        m.root_R[k] = Rr.reshape(9)[k]
    for k in range(3):
        m.root_p[k] = [0.1, -0.2, 1.0][k]
    return m


def test_bias_matches_lagrange_equations_fixed_root():
    """c_i = sum_k dM_ij/dq_k v_j v_k - 1/2 v^T dM/dq_i v + dU/dq_i (hinge
    coordinates are true generalized coordinates when the root is fixed)."""
    rng = np.random.default_rng(7)
    models = [H.brick_chain(4)] + [_fixed_root(m, rng) for m in _small_models()[:6]]
    eps = 1e-6
    for m in models:
        q, v = _random_state(m, rng, ang=1.0)
        n = O.nv(m)
        p = O.default_params()
        dM = np.zeros((n, n, n))
        dU = np.zeros(n)
        for k in range(n):
            e = np.zeros(n)
            e[k] = eps
            dM[k] = (O.mass_matrix(m, q + e, p) - O.mass_matrix(m, q - e, p)) / (2 * eps)
            dU[k] = (H.potential(m, q + e) - H.potential(m, q - e)) / (2 * eps)
        Mdot_v = np.einsum("kij,j,k->i", dM, v, v)
        half_grad = 0.5 * np.einsum("kij,i,j->k", dM, v, v)
        c_lag = Mdot_v - half_grad + dU
        c = O.bias(m, q, v, p)
        assert np.abs(c - c_lag).max() < 1e-6 * max(1.0, np.abs(c_lag).max())


def test_bias_momentum_balance_free_robots():
    """Free robots, no contact, no actuation: the rate of total linear momentum
    is m_tot g and the rate of angular momentum about the world origin is the
    gravity moment.  Momenta come from FK differences; the acceleration is
    M^-1 (-c) from the oracle."""
    rng = np.random.default_rng(9)
    for m in _small_models():
        q, v = _random_state(m, rng)
        p = O.default_params(armature=0.0)
        M = O.mass_matrix(m, q, p)
        c = O.bias(m, q, v, p)
        vdot = np.linalg.solve(M, -c)
        qd = H.qdot_from_v(m, q, v)
        h = 1e-4
        Pp, Lp = H.momentum_fd(m, q + h * qd, v + h * vdot)
        Pm, Lm = H.momentum_fd(m, q - h * qd, v - h * vdot)
        dP = (Pp - Pm) / (2 * h)
        dL = (Lp - Lm) / (2 * h)
        _, _, cc = O.fk(m, q)
        mt = sum(m.mass[b] for b in range(m.nb))
        g = np.array([0.0, 0.0, -G])
        tau_g = sum(np.cross(cc[b], m.mass[b] * g) for b in range(m.nb))
        scale = mt * G * (1 + np.abs(cc).max())
        assert np.abs(dP - mt * g).max() < 2e-5 * scale
        assert np.abs(dL - tau_g).max() < 2e-5 * scale


def test_bias_zero_gravity_rest_is_zero():
    m = O.model_from_population(P.quadrupeds(1), 0)
    q, _ = _random_state(m, np.random.default_rng(3))
    c = O.bias(m, q, np.zeros(O.nv(m)), O.default_params(gravity=(0, 0, 0)))
    assert np.abs(c).max() == 0.0


# ----------------------------------------------------------------- Cholesky
def test_cholesky_residual_and_independent_solve():
    rng = np.random.default_rng(2)
    for n in (1, 6, 14, 26):
        A = rng.normal(size=(n, n))
        M = A @ A.T + n * np.eye(n)
        rc, L = O.cholesky(M)
        assert rc == 0
        assert np.allclose(np.triu(L, 1), 0.0)
        assert np.abs(L @ L.T - M).max() < 1e-12 * np.abs(M).max()
        b = rng.normal(size=n)
        x = np.linalg.solve(L.T, np.linalg.solve(L, b))
        import scipy.linalg as sl
        lu = sl.lu_factor(M)
        assert np.abs(x - sl.lu_solve(lu, b)).max() < 1e-10 * np.abs(x).max()
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    rc, _ = O.cholesky(bad)
    assert rc == -1


# --------------------------------------------------------- hinge dynamics
def test_compound_pendulum_small_angle_period():
    """T = 2 pi sqrt(I_pivot / (m g l)) for a brick hanging from a hinge."""
    m = H.brick_chain(1)
    dt = 1e-4
    mb, h, l = 0.216, 0.03, 0.03
    I_pivot = mb * (2 * h * h) / 3.0 + mb * l * l
    T_exact = 2 * np.pi * np.sqrt(I_pivot / (mb * G * l))
    q, v, s = np.array([0.01]), np.array([0.0]), np.zeros(2)
    p = prm(dt=dt, armature=0.0)
    th = [q[0]]
    chunk = 10
    for _ in range(int(3.2 * T_exact / dt / chunk)):
        q, v, s, st, _ = O.run(m, q, v, s, chunk, prm=p)
        th.append(q[0])
    th = np.array(th)
    t = np.arange(len(th)) * dt * chunk
    up = [i for i in range(1, len(th)) if th[i - 1] < 0 <= th[i]]
    times = [t[i - 1] + (t[i] - t[i - 1]) * (-th[i - 1]) / (th[i] - th[i - 1]) for i in up]
    period = np.diff(times).mean()
    assert abs(period - T_exact) / T_exact < 1e-3


def _chain_energy_drift(dt, steps):
    m = H.brick_chain(5)
    p = prm(dt=dt)
    q = np.array([0.5, 0.3, -0.2, 0.4, 0.1])
    v = np.zeros(5)
    s = np.zeros(10)

    def energy(q, v):
        return 0.5 * v @ O.mass_matrix(m, q, p) @ v + H.potential(m, q)

    E0 = energy(q, v)
    drift = 0.0
    chunk = steps // 50
    for _ in range(50):
        q, v, s, _, _ = O.run(m, q, v, s, chunk, prm=p)
        drift = max(drift, abs(energy(q, v) - E0))
    scale = sum(m.mass[b] for b in range(1, 6)) * G * 0.3
    return drift / scale


def test_chain_energy_drift_bounded_and_first_order():
    """Semi-implicit Euler on a non-separable Hamiltonian: bounded drift that
    shrinks linearly with dt (no contact, no actuation, gravity on)."""
    d1 = _chain_energy_drift(1e-4, 10000)
    d2 = _chain_energy_drift(0.5e-4, 20000)
    assert d1 < 1e-3
    assert 1.5 < d1 / d2 < 2.6


# ---------------------------------------------------------------- contacts
def test_plane_contacts_hand_placed_cube():
    """Cube centre at z = 0.04: the four bottom vertices are 1 cm deep, in
    vertex order (x sign bit 0, y sign bit 1, z sign bit 2)."""
    m = H.single_box()
    c = O.contacts(m, free_q((0.2, 0.1, 0.04)), O.default_params())
    assert len(c["a"]) == 4
    assert np.all(c["b"] == -1)
    assert np.allclose(c["depth"], 0.01, atol=1e-15)
    exp = [[0.15, 0.05, -0.01], [0.25, 0.05, -0.01], [0.15, 0.15, -0.01], [0.25, 0.15, -0.01]]
    assert np.allclose(c["p"], exp, atol=1e-15)
    assert np.allclose(c["n"], [[0, 0, 1]] * 4)
    # tilted: only the single lowest corner is below the plane
    q = free_q((0, 0, 0.08), quat=np.array([np.cos(0.3), np.sin(0.3) * 0.6, np.sin(0.3) * 0.8, 0.0]))
    R, _, _ = O.fk(m, q)
    verts = [q[:3] + R[0] @ (0.05 * np.array([1 if (k >> i) & 1 else -1 for i in range(3)]))
             for k in range(8)]
    zmin = min(v[2] for v in verts)
    q[2] -= zmin + 0.002
    c = O.contacts(m, q, O.default_params())
    assert len(c["a"]) == 1
    assert abs(c["depth"][0] - 0.002) < 1e-14


def _two_free_boxes(pa, Ra, pb, Rb, ha=0.03, hb=0.03):
    """Fixed root far away with two children placed by their joint frames."""
    bodies = [dict(half=(0.05, 0.05, 0.05), mass=1.0),
              dict(parent=0, axis=1, R_fix=Ra, p_fix=pa, half=(ha, ha, ha)),
              dict(parent=0, axis=1, R_fix=Rb, p_fix=pb, half=(hb, hb, hb))]
    return H.make_model(bodies, root_fixed=True, root_p=(0.0, 0.0, 5.0))


def test_box_box_face_face_patch():
    """A small box resting 1 mm into a larger one: four contacts at the small
    box's bottom corners, depth 1 mm, normal from the upper box (b) to the
    lower (a) is -z."""
    d = 0.001
    m = _two_free_boxes((0.0, 1.0, 0.0), np.eye(3), (0.004, 1.003, 0.05 - d), np.eye(3), 0.03, 0.02)
    c = O.contacts(m, np.zeros(2), O.default_params(ground=0))
    assert len(c["a"]) == 4
    assert np.all(c["a"] == 1) and np.all(c["b"] == 2)
    assert np.allclose(c["depth"], d, atol=1e-12)
    assert np.allclose(c["n"], [[0, 0, -1]] * 4, atol=1e-12)
    pts = sorted(map(tuple, np.round(c["p"] - [0, 0, 5.0], 12)))
    exp = sorted((0.004 + sx, 1.003 + sy, 0.03 - d) for sx in (-0.02, 0.02) for sy in (-0.02, 0.02))
    assert np.allclose(pts, exp, atol=1e-12)
    # separated by 1 mm: no contact
    m = _two_free_boxes((0.0, 1.0, 0.0), np.eye(3), (0.004, 1.003, 0.05 + d), np.eye(3), 0.03, 0.02)
    assert len(O.contacts(m, np.zeros(2), O.default_params(ground=0))["a"]) == 0


def _box_vertices(c, R, h):
    return np.array([c + R @ (h * np.array([1 if (k >> i) & 1 else -1 for i in range(3)]))
                     for k in range(8)])


def test_box_box_edge_edge_crossed():
    """Two edges crossing: A is turned 45 deg about y so its top edge runs
    along y; B is turned 45 deg about x so its lowest edge runs along x.
    Expected from the support functions: normal along z, depth = overlap of
    the two edge heights, point midway between the two edges."""
    Ra = H.rot("y", np.pi / 4)
    Rb = H.rot("x", np.pi / 4)
    h = 0.03
    top_a = h * np.sqrt(2)
    d = 0.002
    ca = np.array([0.0, 1.0, 0.0])
    cb = ca + np.array([0.001, -0.002, 2 * top_a - d])
    m = _two_free_boxes(ca, Ra, cb, Rb, h, h)
    c = O.contacts(m, np.zeros(2), O.default_params(ground=0))
    assert len(c["a"]) == 1
    assert np.allclose(np.abs(c["n"][0]), [0, 0, 1], atol=1e-12)
    assert c["n"][0][2] < 0
    assert abs(c["depth"][0] - d) < 1e-12
    # brute-force support overlap along the returned normal
    va = _box_vertices(ca, Ra, h)
    vb = _box_vertices(cb, Rb, h)
    n = -c["n"][0]
    assert abs((va @ n).max() - (vb @ n).min() - c["depth"][0]) < 1e-12
    # contact point: midway between A's top edge (along y at x = ca_x, height
    # top_a) and B's bottom edge (along x at y = cb_y, height cb_z - top_a)
    p = c["p"][0] - [0, 0, 5.0]
    assert np.allclose(p, [ca[0], cb[1], top_a - d / 2], atol=1e-12)


def _two_boxes(pa, Ra, ha, pb, Rb, hb):
    """Fixed root far away with two boxes of any half sizes as its children."""
    bodies = [dict(half=(0.05, 0.05, 0.05), mass=1.0),
              dict(parent=0, axis=1, R_fix=Ra, p_fix=pa, half=tuple(ha)),
              dict(parent=0, axis=1, R_fix=Rb, p_fix=pb, half=tuple(hb))]
    return H.make_model(bodies, root_fixed=True, root_p=(0.0, 0.0, 5.0))


@pytest.mark.parametrize("ratio,face", [(0.93, False), (0.97, True)])
def test_box_box_face_preferred_unless_edge_below_095(ratio, face):
    """The separating-axis choice prefers a face axis unless the best edge
    axis overlaps less than 0.95 x the best face axis.  A plate A (half sizes
    a = (0.01, 0.03, 0.05)) turned 45 deg about y and a cube B (b = 0.03)
    turned 45 deg about x, B straight above A by dz: A's top edge (along y)
    and B's bottom edge (along x) cross, and by the support functions
      edge axis z:      e = (a1 + a3 + b2 + b3)/sqrt2 - dz,
      face axis A_x:    f = a1 + b1/sqrt2 + (b2 + b3)/2 - dz/sqrt2,
    the smallest edge and face overlaps (every other axis overlaps by more
    than 2 cm).  dz is solved for e = ratio * f; the edge overlap is the
    smaller of the two in both cases.  Below 0.95 the pair gives the
    edge-edge point (one contact, normal -z, depth e); above it the face case
    (normal A_x from B to A, deepest point exactly f)."""
    c = np.sqrt(0.5)
    a = np.array([0.01, 0.03, 0.05])
    b = np.array([0.03, 0.03, 0.03])
    K = (a[0] + a[2] + b[1] + b[2]) * c
    F0 = a[0] + c * b[0] + (b[1] + b[2]) / 2
    dz = (K - ratio * F0) / (1 - ratio * c)
    e, f = K - dz, F0 - c * dz
    assert e < f and abs(e / f - ratio) < 1e-12
    Ra, Rb = H.rot("y", np.pi / 4), H.rot("x", np.pi / 4)
    ca = np.array([0.0, 1.0, 0.0])
    m = _two_boxes(ca, Ra, a, ca + np.array([0.0, 0.0, dz]), Rb, b)
    cl = O.contacts(m, np.zeros(2), O.default_params(ground=0))
    if face:
        assert len(cl["a"]) >= 1
        assert np.allclose(cl["n"], [Ra[:, 0]] * len(cl["a"]), atol=1e-12)
        assert abs(cl["depth"].max() - f) < 1e-12
    else:
        assert len(cl["a"]) == 1
        assert np.allclose(cl["n"][0], [0.0, 0.0, -1.0], atol=1e-12)
        assert abs(cl["depth"][0] - e) < 1e-12


def test_box_box_separation_agrees_with_point_sampling():
    """SAT verdicts against Monte-Carlo: a separated pair has no sample point
    inside both boxes; a pair reported 5 mm deep has some."""
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, size=(40000, 3))
    checked = [0, 0]
    for _ in range(60):
        Ra = H.rot("z", rng.uniform(0, 6)) @ H.rot("x", rng.uniform(0, 6))
        Rb = H.rot("y", rng.uniform(0, 6)) @ H.rot("z", rng.uniform(0, 6))
        ca = np.array([0.0, 1.0, 0.0])
        cb = ca + rng.normal(0, 0.035, 3)
        m = _two_free_boxes(ca, Ra, cb, Rb)
        c = O.contacts(m, np.zeros(2), O.default_params(ground=0))
        pts = ca + (Ra @ (0.03 * u).T).T
        loc = (Rb.T @ (pts - cb).T).T
        inside_both = np.any(np.all(np.abs(loc) <= 0.03, axis=1))
        if len(c["a"]) == 0:
            assert not inside_both
            checked[0] += 1
        elif c["depth"].max() > 0.005:
            assert inside_both
            checked[1] += 1
    assert checked[0] > 5 and checked[1] > 5


def test_contact_cap_keeps_deepest_in_list_order():
    rng = np.random.default_rng(0)
    m = H.single_box()
    q = free_q((0, 0, 0.03))           # 4 vertices 2 cm deep
    c4 = O.contacts(m, q, O.default_params())
    q = free_q((0, 0, 0.03), quat=np.array([1.0, 0.02, 0.01, 0.0]) / np.linalg.norm([1.0, 0.02, 0.01, 0.0]))
    c = O.contacts(m, q, O.default_params(contact_cap=2))
    assert c["status"] & O.ST_OVERFLOW
    call = O.contacts(m, q, O.default_params())
    order = np.argsort(-call["depth"], kind="stable")[:2]
    assert np.allclose(c["depth"], call["depth"][np.sort(order)])
    assert len(c4["a"]) == 4


# -------------------------------------------------------------------- PGS
def _tilted_single_corner(depth=0.001):
    m = H.single_box()
    quat = np.array([np.cos(0.3), np.sin(0.3) * 0.6, np.sin(0.3) * 0.8, 0.0])
    q = free_q((0.0, 0.0, 0.08), quat=quat)
    R, _, _ = O.fk(m, q)
    verts = [R[0] @ (0.05 * np.array([1 if (k >> i) & 1 else -1 for i in range(3)])) for k in range(8)]
    k = int(np.argmin([v[2] for v in verts]))
    q[2] = -verts[k][2] - depth
    return m, q, verts[k]


def test_pgs_single_frictionless_contact_closed_form():
    """One contact, mu = 0: Gauss-Seidel converges in one sweep to
    lambda = max(0, (t - J v_free) / (A + R)), and afterwards the soft
    constraint J v+ - t + R lambda = 0 holds; t = min(ERP depth / dt,
    max_correct_vel) (below and above the cap)."""
    _single_contact_case(0.0004, capped=False)
    _single_contact_case(0.003, capped=True)


def _single_contact_case(depth, capped):
    m, q, corner = _tilted_single_corner(depth)
    v = np.array([0.1, -0.05, -0.5, 0.3, -0.2, 0.1])
    p = O.default_params(mu=0.0)
    d = O.step_detail(m, q, v, np.zeros(2), prm=p)
    assert d["nc"] == 1
    # J of the corner point along +z, by finite differences of FK
    n = O.nv(m)
    J = np.zeros(n)
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        qd = H.qdot_from_v(m, q, e)
        Rp, pp, _ = O.fk(m, q + eps * qd)
        Rm, pm, _ = O.fk(m, q - eps * qd)
        local = O.fk(m, q)[0][0].T @ corner
        xp = pp[0] + Rp[0] @ local
        xm = pm[0] + Rm[0] @ local
        J[i] = (xp[2] - xm[2]) / (2 * eps)
    M = O.mass_matrix(m, q, p)
    c = O.bias(m, q, v, p)
    vfree = v + p.dt * np.linalg.solve(M, -c)
    assert np.allclose(d["vfree"], vfree, atol=1e-12)
    A = J @ np.linalg.solve(M, J)
    omg = 2 * np.pi / p.soft_tau
    kden = p.dt * omg * omg + 2 * p.soft_zeta * omg
    erp = p.dt * omg * omg / kden
    kappa = 1.0 / (p.dt * kden)
    t = erp * depth / p.dt
    assert (t > p.max_correct_vel) == capped
    t = min(t, p.max_correct_vel)
    lam = max(0.0, (t - J @ vfree) / (A + kappa * A))
    assert abs(d["lam"][0, 0] - lam) < 1e-8 * max(lam, 1e-3)
    assert np.allclose(d["lam"][0, 1:], 0.0)
    assert abs(J @ d["v"][:n] - t + kappa * A * lam) < 1e-8
    # one sweep and thirty sweeps agree for a single frictionless contact
    d1 = O.step_detail(m, q, v, np.zeros(2), prm=O.default_params(mu=0.0, pgs_iters=1))
    assert np.allclose(d1["v"], d["v"], atol=1e-13)


def _vertices_world(m, q):
    R, p, _ = O.fk(m, q)
    out = []
    for b in range(m.nb):
        for k in range(8):
            loc = np.array(m.com[b][:]) + np.array([1 if (k >> i) & 1 else -1 for i in range(3)]) * np.array(m.half[b][:])
            out.append((b, loc, p[b] + R[b] @ loc))
    return out


def test_pgs_single_contact_on_a_hinged_brick():
    """A brick on a hinge dips one corner 1 mm into the plane; mu = 0.  The
    Jacobian of that corner (finite differences of FK, hinge column included)
    gives lambda = max(0, (t - J v_free) / (A + R)) after one sweep."""
    m = H.make_model([dict(half=(0.05, 0.05, 0.05), mass=1.0),
                      dict(parent=0, axis=1, p_fix=(0.05, 0, 0), com=(0.03, 0, 0))])
    q = free_q((0.0, 0.0, 0.3), quat=np.array([1.0, 0.05, 0.02, 0.0]) / np.linalg.norm([1.0, 0.05, 0.02, 0.0]),
               hinges=[0.9])
    verts = _vertices_world(m, q)
    zs = [x[2][2] for x in verts]
    k = int(np.argmin(zs))
    assert verts[k][0] == 1 and sorted(zs)[1] - zs[k] > 0.005
    q[2] -= zs[k] + 0.001
    body, local, _ = verts[k]
    v = np.array([0.05, 0.02, -0.3, 0.2, -0.4, 0.1, -1.5])
    p = O.default_params(mu=0.0, box_box=0)
    d = O.step_detail(m, q, v, np.zeros(2 * O.MAXB), prm=p)
    assert d["nc"] == 1
    n = O.nv(m)
    J = np.zeros(n)
    eps = 1e-7
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        qd = H.qdot_from_v(m, q, e)
        Rp, pp, _ = O.fk(m, q + eps * qd)
        Rm, pm, _ = O.fk(m, q - eps * qd)
        J[i] = ((pp[body] + Rp[body] @ local)[2] - (pm[body] + Rm[body] @ local)[2]) / (2 * eps)
    assert abs(J[6]) > 0.01
    M = O.mass_matrix(m, q, p)
    vfree = d["vfree"]
    A = J @ np.linalg.solve(M, J)
    omg = 2 * np.pi / p.soft_tau
    kden = p.dt * omg * omg + 2 * p.soft_zeta * omg
    erp = p.dt * omg * omg / kden
    kappa = 1.0 / (p.dt * kden)
    t = min(erp * 0.001 / p.dt, p.max_correct_vel)
    lam = max(0.0, (t - J @ vfree) / (A + kappa * A))
    assert lam > 0
    assert abs(d["lam"][0, 0] - lam) < 1e-7 * lam
    assert abs(J @ d["v"][:n] - t + kappa * A * lam) < 1e-8


def test_internal_contact_impulses_conserve_momentum():
    """Box/box contacts inside one robot exchange equal and opposite impulses:
    the contact part of the velocity change, M (v+ - v_free), has no net
    linear or angular momentum (rows 0..5 of a free root)."""
    g = P.grammar(40, seed=3)
    p = O.default_params(ground=0, gravity=(0, 0, 0), actuate=0)
    rng = np.random.default_rng(1)
    seen = 0
    for i in range(g.n):
        m = O.model_from_population(g, i)
        n = O.nv(m)
        q = g.q0[i, :O.nq(m)].copy()
        q[7:] = rng.uniform(-1.2, 1.2, n - 6)
        v = np.zeros(n)
        d = O.step_detail(m, q, v, np.zeros(2 * O.MAXB), prm=p)
        if d["nc"] == 0 or np.abs(d["lam"]).max() < 1e-6:
            continue
        seen += 1
        M = O.mass_matrix(m, q, p)
        dp = M @ (d["v"][:n] - d["vfree"])
        assert np.abs(dp[:6]).max() < 1e-12 * max(1.0, np.abs(dp).max())
        assert np.abs(dp[6:]).max() > 1e-6
    assert seen >= 3


def test_zero_jacobian_row_is_frozen():
    """A planar mechanism (fixed root, every hinge about y) pressing an edge
    1 mm into the ground: the ground tangent along y has J = 0 (no dof moves
    the contact points along y), so that row is frozen -- its impulse stays
    exactly 0 -- while the normal and x rows carry impulses.  The same kind of
    mechanism colliding with itself (a contact whose tangent plane holds the
    direction no dof can move) keeps the step finite."""
    q = np.array([0.3, 0.2])
    m0 = H.brick_chain(2, root_fixed=True, root_p=(0.0, 0.0, 0.2))
    R, p, c = O.fk(m0, q)
    low = min((c[b] + R[b] @ (np.array([sx, sy, sz]) * np.array(m0.half[b][:])))[2]
              for b in range(m0.nb) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1))
    m = H.brick_chain(2, root_fixed=True, root_p=(0.0, 0.0, 0.2 - low - 0.001))
    cl = O.contacts(m, q, O.default_params())
    assert len(cl["a"]) == 2 and np.all(cl["b"] == -1) and np.allclose(cl["depth"], 0.001, atol=1e-12)
    for v in (np.array([1.0, 1.0]), np.array([-1.0, -1.0])):
        d = O.step_detail(m, q, v, np.zeros(2 * O.MAXB), prm=O.default_params(actuate=0))
        assert d["status"] == 0 and np.all(np.isfinite(d["v"]))
        assert np.all(d["lam"][:, 2] == 0.0)
        assert np.all(d["lam"][:, 0] > 0.0) and np.all(np.abs(d["lam"][:, 1]) > 0.0)
    # self-collision of a planar mechanism (all hinges about x)
    Rb1 = np.array([[0, -1, 0], [0, 0, 1], [-1, 0, 0]], float)
    Rb2 = np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 1]], float)
    m = H.make_model([dict(half=(0.05, 0.05, 0.05), mass=1.0, exclude=0b110),
                      dict(parent=0, R_fix=Rb1, p_fix=(0, 0, -0.05), com=(0.03, 0, 0), exclude=0b1001),
                      dict(parent=0, R_fix=Rb2, p_fix=(0, -0.05, 0), com=(0.03, 0, 0), exclude=0b1),
                      dict(parent=1, R_fix=np.diag([1.0, -1.0, -1.0]), p_fix=(0.06, 0, 0), com=(0.03, 0, 0),
                           exclude=0b10)])
    quat = np.array([0.9977, 0.06772, 0.0, 0.0])
    q = free_q((0.0, 0.0032, 0.16636), quat=quat / np.linalg.norm(quat), hinges=[0.86087, 0.92013, 0.96376])
    v = np.array([0.0, 0.02, -0.47, 5.0, 0.0, 0.0, 18.7, 13.9, 5.5])
    c = O.contacts(m, q, O.default_params())
    assert any(a == 1 and b == 2 for a, b in zip(c["a"], c["b"]))
    d = O.step_detail(m, q, v, np.zeros(2 * O.MAXB))
    assert d["status"] == 0 and np.all(np.isfinite(d["v"]))
    k = [j for j in range(d["nc"]) if c["b"][j] == 2][0]
    assert c["n"][k][0] == 0.0 and d["lam"][k, 0] > 0.0


def test_resting_cube_steady_penetration():
    """Resting flat cube: per-contact impulse m g dt / 4 and steady depth
    d* = kappa A lambda dt / ERP, with A = 1/m + |r x n|^2 / I for a corner."""
    m = H.single_box()
    p = O.default_params()
    q = free_q((0.0, 0.0, 0.0501))
    v = np.zeros(6)
    q, v, _, st, _ = O.run(m, q, v, np.zeros(2), 3000, prm=p)
    omg = 2 * np.pi / p.soft_tau
    kden = p.dt * omg * omg + 2 * p.soft_zeta * omg
    erp = p.dt * omg * omg / kden
    kappa = 1.0 / (p.dt * kden)
    I = 1.0 * 0.1 ** 2 / 6
    A = 1.0 + (0.05 ** 2 + 0.05 ** 2) / I
    lam = 1.0 * G * p.dt / 4
    dstar = kappa * A * lam * p.dt / erp
    assert st == 0
    assert abs(q[2] - (0.05 - dstar)) < 1e-6
    assert np.abs(v).max() < 1e-6


def test_heavy_cube_rests_on_the_softness_floor():
    """100 kg cube of the same size: kappa A = kappa * 4 / 100 < min_cfm, so
    the floored softness R = min_cfm sets the steady depth d* = min_cfm
    lambda dt / ERP (lambda = m g dt / 4 per corner), four times the depth
    kappa A would give; the recovery speed ERP d* / dt stays below the cap."""
    m = H.single_box(mass=100.0)
    p = O.default_params()
    q = free_q((0.0, 0.0, 0.0501))
    v = np.zeros(6)
    q, v, _, st, _ = O.run(m, q, v, np.zeros(2), 4000, prm=p)
    omg = 2 * np.pi / p.soft_tau
    kden = p.dt * omg * omg + 2 * p.soft_zeta * omg
    erp = p.dt * omg * omg / kden
    kappa = 1.0 / (p.dt * kden)
    I = 100.0 * 0.1 ** 2 / 6
    A = 1.0 / 100.0 + (0.05 ** 2 + 0.05 ** 2) / I
    assert kappa * A < p.min_cfm
    lam = 100.0 * G * p.dt / 4
    dstar = p.min_cfm * lam * p.dt / erp
    assert erp * dstar / p.dt < p.max_correct_vel
    assert st == 0
    assert abs(q[2] - (0.05 - dstar)) < 1e-6
    assert abs(dstar - kappa * A * lam * p.dt / erp) > 1e-4  # the floor, not kappa A, decides
    assert np.abs(v).max() < 1e-6


@pytest.mark.parametrize("alpha_deg,slides", [(20.0, False), (35.0, True)])
def test_incline_stick_slide(alpha_deg, slides):
    """Tilted gravity on a flat plane = an incline: with mu = 0.5 the cube
    sticks (only soft-friction creep) iff tan(alpha) <= mu, else it slides
    with deceleration g (sin a - mu cos a)."""
    a = np.radians(alpha_deg)
    p = O.default_params(mu=0.5, gravity=(G * np.sin(a), 0.0, -G * np.cos(a)))
    m = H.single_box()
    q = free_q((0.0, 0.0, 0.0499))
    v = np.zeros(6)
    q, v, _, _, _ = O.run(m, q, v, np.zeros(2), 100, prm=p)
    v_before = v[0]
    q, v, _, _, _ = O.run(m, q, v, np.zeros(2), 400, prm=p)
    if slides:
        acc = (v[0] - v_before) / (400 * p.dt)
        assert abs(acc - G * (np.sin(a) - 0.5 * np.cos(a))) < 0.01 * G * np.sin(a)
    else:
        assert abs(v[0]) < 0.02
        assert abs(q[0]) < 0.02


def _rot_of_quat(qq):
    w, x, y, z = qq
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_asymmetric_box_spin_conserves_momentum_and_flips():
    """Torque-free spin of a box with three different moments, started near
    its intermediate axis: world angular momentum and kinetic energy are
    invariants of Euler's equations (kept to the explicit integrator's drift,
    measured 0.6 % and 1.1 % over 8 s), and rotation about the intermediate
    axis is unstable, so the spin flips (the body-axis rate changes sign)."""
    h = np.array([0.05, 0.03, 0.015])
    m = H.make_model([dict(half=tuple(h), mass=1.0)])
    p = prm(gravity=(0.0, 0.0, 0.0))
    I = np.array([h[1] ** 2 + h[2] ** 2, h[0] ** 2 + h[2] ** 2, h[0] ** 2 + h[1] ** 2]) / 3.0
    q = free_q((0.0, 0.0, 1.0))
    v = np.array([0.0, 0.0, 0.0, 0.01, 5.0, 0.01])
    L0 = _rot_of_quat(q[3:7]) @ (I * v[3:6])
    E0 = 0.5 * np.sum(I * v[3:6] ** 2)
    wy = []
    for _ in range(40):
        q, v, _, st, _ = O.run(m, q, v, np.zeros(2), 100, prm=p)
        L = _rot_of_quat(q[3:7]) @ (I * v[3:6])
        assert np.linalg.norm(L - L0) <= 0.02 * np.linalg.norm(L0)
        assert abs(0.5 * np.sum(I * v[3:6] ** 2) - E0) <= 0.03 * E0
        wy.append(v[4])
    assert st == 0 and min(wy) < -4.5 and max(wy) > 4.5


# ------------------------------------------------------------------ spheres
def test_sphere_plane_contact_hand_placed():
    """A tilted free ball whose centre sits off its frame origin: one contact
    at the centre's foot, r below it, depth r - z_centre, normal +z; lifted
    by 2 mm, none."""
    R = H.rot("x", 0.7) @ H.rot("z", 0.3)
    quat = _quat_of(R)
    com = np.array([0.01, -0.02, 0.005])
    m = H.single_ball(0.05, 1.0, com=tuple(com))
    p0 = np.array([0.3, -0.2, 0.0])
    centre = p0 + R @ com
    p0[2] += 0.049 - centre[2]
    centre = p0 + R @ com
    c = O.contacts(m, free_q(tuple(p0), tuple(quat)), O.default_params())
    assert len(c["a"]) == 1 and c["a"][0] == 0 and c["b"][0] == -1
    assert abs(c["depth"][0] - 0.001) < 1e-12
    assert np.allclose(c["n"][0], [0, 0, 1])
    assert np.allclose(c["p"][0], centre - [0, 0, 0.05], atol=1e-12)
    p0[2] += 0.002
    assert len(O.contacts(m, free_q(tuple(p0), tuple(quat)), O.default_params())["a"]) == 0


def _quat_of(R):
    """Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's method)."""
    t = np.trace(R)
    if t > 0:
        w = np.sqrt(1 + t) / 2
        return np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])
    i = int(np.argmax(np.diag(R)))
    j, k = (i + 1) % 3, (i + 2) % 3
    x = np.sqrt(1 + R[i, i] - R[j, j] - R[k, k]) / 2
    q = np.zeros(4)
    q[0] = (R[k, j] - R[j, k]) / (4 * x)
    q[1 + i] = x
    q[1 + j] = (R[j, i] + R[i, j]) / (4 * x)
    q[1 + k] = (R[k, i] + R[i, k]) / (4 * x)
    return q


def test_resting_ball_steady_penetration():
    """A ball at rest has one contact straight below its centre, so the row
    has A = 1/m (no lever arm), impulse m g dt and steady depth
    d* = kappa A lambda dt / ERP."""
    mass = 1000.0 * 4.0 / 3.0 * np.pi * 0.05 ** 3
    m = H.single_ball(0.05, mass)
    p = O.default_params()
    q, v, _, st, _ = O.run(m, free_q((0.0, 0.0, 0.0501)), np.zeros(6), np.zeros(2), 3000, prm=p)
    omg = 2 * np.pi / p.soft_tau
    kden = p.dt * omg * omg + 2 * p.soft_zeta * omg
    erp = p.dt * omg * omg / kden
    kappa = 1.0 / (p.dt * kden)
    A = 1.0 / mass
    assert kappa * A > p.min_cfm
    lam = mass * G * p.dt
    dstar = kappa * A * lam * p.dt / erp
    assert st == 0
    assert abs(q[2] - (0.05 - dstar)) < 1e-7
    assert np.abs(v).max() < 1e-6


@pytest.mark.parametrize("alpha_deg,mu,rolls", [(20.0, 0.5, True), (40.0, 0.1, False)])
def test_ball_on_incline_rolls_or_slides(alpha_deg, mu, rolls):
    """Tilted gravity on a flat plane = an incline.  A solid ball (I = 2/5 m r^2)
    rolls without slipping iff mu >= (2/7) tan(alpha), with acceleration
    (5/7) g sin(alpha) and v = omega r; otherwise it slides with acceleration
    g (sin a - mu cos a) while friction spins it up at 5 mu g cos(a) / (2 r).
    A wrong moment of inertia, lever arm or contact point fails both."""
    a = np.radians(alpha_deg)
    r = 0.05
    assert (mu >= 2.0 / 7.0 * np.tan(a)) == rolls
    p = O.default_params(mu=mu, gravity=(G * np.sin(a), 0.0, -G * np.cos(a)))
    m = H.single_ball(r, 0.5)
    q = free_q((0.0, 0.0, r - 1e-4))
    q, v, _, _, _ = O.run(m, q, np.zeros(6), np.zeros(2), 100, prm=p)
    v0, w0 = v[0], v[4]
    t = 400 * p.dt
    q, v, _, st, _ = O.run(m, q, v, np.zeros(2), 400, prm=p)
    assert st == 0
    acc = (v[0] - v0) / t
    spin = (v[4] - w0) / t   # body y spin, world y while the ball turns about y
    if rolls:
        assert abs(acc - 5.0 / 7.0 * G * np.sin(a)) < 0.01 * G * np.sin(a)
        assert abs(v[0] - v[4] * r) < 0.01 * abs(v[0])
    else:
        assert abs(acc - G * (np.sin(a) - mu * np.cos(a))) < 0.01 * G * np.sin(a)
        assert abs(spin - 5.0 * mu * G * np.cos(a) / (2.0 * r)) < 0.01 * 5.0 * mu * G * np.cos(a) / (2.0 * r)
        assert v[0] - v[4] * r > 0.1


def _ball_and_box(pa, Ra, pb, Rb, ga, gb, ha=0.03, hb=0.03):
    """Fixed root far away with two children (geometry ga, gb) placed by their
    joint frames; both centred on their frame origins."""
    bodies = [dict(half=(0.05, 0.05, 0.05), mass=1.0),
              dict(parent=0, axis=1, R_fix=Ra, p_fix=pa, half=(ha, ha, ha), geom=ga),
              dict(parent=0, axis=1, R_fix=Rb, p_fix=pb, half=(hb, hb, hb), geom=gb)]
    return H.make_model(bodies, root_fixed=True, root_p=(0.0, 0.0, 5.0))


def _box_surface(c, R, h, k=120):
    """Points on a box's surface, k x k per face."""
    g = np.linspace(-1.0, 1.0, k)
    u, w = np.meshgrid(g, g)
    u, w = u.ravel(), w.ravel()
    pts = []
    for ax in range(3):
        for sg in (-1.0, 1.0):
            loc = np.zeros((u.size, 3))
            loc[:, ax] = sg
            loc[:, (ax + 1) % 3] = u
            loc[:, (ax + 2) % 3] = w
            pts.append(loc * h)
    return c + np.concatenate(pts) @ R.T


def test_sphere_sphere_contact_against_sampling():
    """Two balls: a contact iff sampled points of one lie inside the other;
    the depth is the overlap of their extents along the returned normal (a
    support-function check), the normal is unit, and the point lies on the
    centre line midway between the two surfaces."""
    rng = np.random.default_rng(11)
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    u *= rng.uniform(0, 1, size=(20000, 1)) ** (1 / 3)
    seen = [0, 0]
    for _ in range(40):
        ca = np.array([0.0, 1.0, 0.0])
        cb = ca + rng.normal(0, 0.035, 3)
        ra, rb = 0.03, rng.uniform(0.015, 0.03)
        m = _ball_and_box(ca, np.eye(3), cb, H.rot("z", 1.0), 1, 1, 0.03, rb)
        c = O.contacts(m, np.zeros(2), O.default_params(ground=0))
        overlap = np.any(np.linalg.norm(ca + ra * u - cb, axis=1) <= rb)
        if len(c["a"]) == 0:
            assert not overlap
            seen[0] += 1
            continue
        assert len(c["a"]) == 1 and (c["a"][0], c["b"][0]) == (1, 2)
        n = c["n"][0]
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        # support functions along n (from b towards a): a reaches down to
        # ca.n - ra, b reaches up to cb.n + rb
        assert abs((cb @ n + rb) - (ca @ n - ra) - c["depth"][0]) < 1e-12
        assert np.allclose(np.cross(n, ca - cb), 0, atol=1e-12) and n @ (ca - cb) > 0
        mid = 0.5 * ((ca + [0, 0, 5.0] - ra * n) + (cb + [0, 0, 5.0] + rb * n))
        assert np.allclose(c["p"][0], mid, atol=1e-12)
        if c["depth"][0] > 0.003:
            assert overlap
        seen[1] += 1
    assert seen[0] > 5 and seen[1] > 5


@pytest.mark.parametrize("ball_first", [True, False])
def test_sphere_box_contact_against_surface_sampling(ball_first):
    """Ball against a rotated box, centre outside and inside the box.  The
    distance from the centre to the box surface, found by sampling the six
    faces densely, gives the depth (r - distance outside, r + distance
    inside) and, through the nearest sample, the normal's direction; the
    normal always points from the higher-index body to the lower."""
    rng = np.random.default_rng(12 if ball_first else 13)
    hb = np.array([0.03, 0.02, 0.025])
    r = 0.02
    seen = [0, 0, 0]
    for _ in range(40):
        Rx = H.rot("z", rng.uniform(0, 6)) @ H.rot("x", rng.uniform(0, 6))
        cx = np.array([0.0, 1.0, 0.0])
        cs = cx + rng.normal(0, 0.03, 3)
        if ball_first:
            m = _ball_and_box(cs, np.eye(3), cx, Rx, 1, 0, r, 0.03)
        else:
            m = _ball_and_box(cx, Rx, cs, np.eye(3), 0, 1, 0.03, r)
        for b in (1, 2):
            if m.geom[b] == 0:
                for k in range(3):
                    m.half[b][k] = hb[k]
        c = O.contacts(m, np.zeros(2), O.default_params(ground=0))
        surf = _box_surface(cx, Rx, hb)
        dist = np.linalg.norm(surf - cs, axis=1)
        j = int(np.argmin(dist))
        inside = np.all(np.abs(Rx.T @ (cs - cx)) <= hb)
        depth = r + dist[j] if inside else r - dist[j]
        if len(c["a"]) == 0:
            assert depth < 1e-3
            seen[0] += 1
            continue
        assert len(c["a"]) == 1 and (c["a"][0], c["b"][0]) == (1, 2)
        assert abs(c["depth"][0] - depth) < 1e-3
        n = c["n"][0]
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        out_dir = (cs - surf[j]) / dist[j] * (-1.0 if inside else 1.0)  # box -> ball
        n_box_to_ball = n if ball_first else -n
        if dist[j] > 0.004:  # the sample grid (0.5 mm) blurs directions closer in
            assert n_box_to_ball @ out_dir > 0.98
        # the point lies between the box surface and the ball's deepest point
        p = c["p"][0] - [0, 0, 5.0]
        deepest = cs - r * n_box_to_ball
        assert np.linalg.norm(p - 0.5 * (deepest + surf[j])) < 2e-3
        seen[2 if inside else 1] += 1
    assert seen[0] > 3 and seen[1] > 5 and seen[2] > 2


def test_ball_modules_keep_momentum_in_free_flight():
    """A grammar robot with ball modules in free flight (gravity off, no
    contacts): linear momentum stays zero-change and the ball's own spin
    about its hinge costs no energy beyond the integrator's drift."""
    pop = P.grammar(40, seed=21, ball_p=0.5)
    i = int(np.argmax([(pop.geom[k] == 1).sum() for k in range(pop.n)]))
    assert (pop.geom[i] == 1).sum() >= 2
    m = O.model_from_population(pop, i)
    assert m.geom[0] == 0 and sum(m.geom[b] for b in range(m.nb)) >= 2
    p = prm(gravity=(0.0, 0.0, 0.0))
    q, v, s = P.random_state(pop.subset([i]), seed=5)
    nq, nv = O.nq(m), O.nv(m)
    q0, v0 = q[0, :nq].copy(), v[0, :nv].copy()
    M0 = O.mass_matrix(m, q0, p)
    e0 = 0.5 * v0 @ M0 @ v0
    q1, v1, _, st, _ = O.run(m, q0, v0, s[0], 200, prm=p)
    assert st == 0
    e1 = 0.5 * v1 @ O.mass_matrix(m, q1, p) @ v1
    assert abs(e1 - e0) < 0.02 * e0


# ---------------------------------------------------------------------- CPG
def test_cpg_single_oscillator_norm_growth():
    """Explicit Euler of a 2x2 rotation generator: |s_n| = |s_0| (1 + dt^2 w^2)^(n/2)."""
    m = H.make_model([dict(half=(0.05, 0.05, 0.05), mass=1.0),
                      dict(parent=0, axis=1, p_fix=(0.05, 0, 0), com=(0.03, 0, 0))],
                     w_int=[0.0, 0.7], w_cpl=[0.0, 0.0])
    p = O.default_params(ground=0, box_box=0, actuate=1, gravity=(0, 0, 0))
    s0 = np.zeros(2 * O.MAXB)
    s0[0:2] = [0.6, -0.3]
    n = 500
    q, v, s, st, _ = O.run(m, free_q((0, 0, 1), hinges=[0.0]), np.zeros(7), s0, n, prm=p)
    growth = (1 + (p.dt * 0.7) ** 2) ** (n / 2)
    assert abs(np.linalg.norm(s[:2]) - np.linalg.norm(s0[:2]) * growth) < 1e-13
    assert abs(np.arctan2(s[1], s[0]) - np.arctan2(s0[1], s0[0]) + n * np.arctan(p.dt * 0.7)) < 1e-10


def test_cpg_generator_is_antisymmetric():
    """(s_{n+1} - s_n) . s_n = 0 for every state iff W is antisymmetric."""
    pop = P.grammar(6, seed=21)
    rng = np.random.default_rng(0)
    p = O.default_params(ground=0, box_box=0, gravity=(0, 0, 0))
    for i in range(pop.n):
        m = O.model_from_population(pop, i)
        nh = m.nb - 1
        s0 = np.zeros(2 * O.MAXB)
        s0[: 2 * nh] = rng.normal(size=2 * nh)
        q0 = pop.q0[i, :O.nq(m)].copy()
        q0[2] += 1.0
        _, _, s1, _, _ = O.run(m, q0, np.zeros(O.nv(m)), s0, 1, prm=p)
        ds = s1[: 2 * nh] - s0[: 2 * nh]
        assert abs(ds @ s0[: 2 * nh]) < 1e-15 * np.linalg.norm(s0) ** 2
        assert np.linalg.norm(ds) > 1e-4


def test_pd_torque_saturates_and_drives_towards_target():
    """Zero gravity, one hinge: a large target error saturates the torque at
    tau_max, so the first-step hinge acceleration equals tau_max / M_hh-ish
    sign: the hinge moves towards the CPG target."""
    m = H.make_model([dict(half=(0.05, 0.05, 0.05), mass=1.0),
                      dict(parent=0, axis=1, p_fix=(0.05, 0, 0), com=(0.03, 0, 0))],
                     w_int=[0.0, 0.0], w_cpl=[0.0, 0.0])
    p = O.default_params(ground=0, box_box=0, actuate=1, gravity=(0, 0, 0))
    s0 = np.zeros(2 * O.MAXB)
    s0[0] = 1.0                      # target theta_max * 1 = pi/2
    q0 = free_q((0, 0, 1), hinges=[0.0])
    q, v, _, _, _ = O.run(m, q0, np.zeros(7), s0, 1, prm=p)
    M = O.mass_matrix(m, q0, p)
    tau = np.zeros(7)
    tau[6] = p.tau_max              # kp * pi/2 = 3.14 > tau_max
    assert np.allclose(v, p.dt * np.linalg.solve(M, tau), atol=1e-14)


# ----------------------------------------------------------------- fitness
def test_fitness_is_core_xy_displacement():
    m = H.single_box()
    q0 = free_q((0.2, -0.1, 5.0))
    q, _, _, _, _ = O.run(m, q0, np.array([0.3, 0.4, 0, 0, 0, 0]), np.zeros(2), 100,
                          prm=prm(gravity=(0, 0, 0)))
    assert abs(O.fitness(q0, q)[0] - 0.5 * 100 * 0.002) < 1e-12
