"""Hand-built model descriptions for the oracle pins (test helpers only)."""
import numpy as np

from oracle import oracle as O


def rot(axis: str, ang: float) -> np.ndarray:
    c, s = np.cos(ang), np.sin(ang)
    if axis == "x":
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == "y":
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def make_model(bodies, root_fixed=False, root_R=None, root_p=(0.0, 0.0, 0.0), w_int=None, w_cpl=None):
    """bodies: list of dicts with parent, axis, R_fix, p_fix, half, com, mass."""
    m = O.Model()
    m.nb = len(bodies)
    m.root_fixed = 1 if root_fixed else 0
    for b in range(O.MAXB):
        m.parent[b] = -1
        for k in range(9):
            m.R_fix[b][k] = 1.0 if k in (0, 4, 8) else 0.0
    for b, d in enumerate(bodies):
        m.parent[b] = d.get("parent", -1)
        m.axis[b] = d.get("axis", 1)
        m.exclude[b] = d.get("exclude", 0)
        Rf = np.asarray(d.get("R_fix", np.eye(3)), dtype=float).reshape(9)
        for k in range(9):
            m.R_fix[b][k] = Rf[k]
        for k in range(3):
            m.p_fix[b][k] = d.get("p_fix", (0, 0, 0))[k]
            m.half[b][k] = d.get("half", (0.03, 0.03, 0.03))[k]
            m.com[b][k] = d.get("com", (0, 0, 0))[k]
        m.mass[b] = d.get("mass", 0.216)
        m.geom[b] = d.get("geom", 0)
        if w_int is not None:
            m.w_int[b] = w_int[b]
        if w_cpl is not None:
            m.w_cpl[b] = w_cpl[b]
    R = np.eye(3) if root_R is None else np.asarray(root_R)
    for k in range(9):
        m.root_R[k] = R.reshape(9)[k]
    for k in range(3):
        m.root_p[k] = root_p[k]
    return m


def single_box(half=0.05, mass=1.0):
    return make_model([dict(half=(half, half, half), mass=mass)])


def single_ball(radius=0.05, mass=1.0, com=(0.0, 0.0, 0.0)):
    """A free solid sphere (geometry 1): radius in half[0], centre at com."""
    return make_model([dict(half=(radius, radius, radius), mass=mass, com=com, geom=1)])


def brick_chain(n_links, root_fixed=True, root_p=(0.0, 0.0, 2.0)):
    """Core cube with a chain of bricks hanging from its -z face.

    Each brick's frame x points down the chain; hinge axis (child y) is
    horizontal.  Consecutive bricks attach at the previous brick's far face.
    """
    down = np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], dtype=float)  # x -> -z
    bodies = [dict(half=(0.05, 0.05, 0.05), mass=1.0)]
    for k in range(n_links):
        if k == 0:
            bodies.append(dict(parent=0, axis=1, R_fix=down, p_fix=(0, 0, -0.05),
                               com=(0.03, 0, 0), half=(0.03, 0.03, 0.03), mass=0.216))
        else:
            bodies.append(dict(parent=k, axis=1, R_fix=np.eye(3), p_fix=(0.06, 0, 0),
                               com=(0.03, 0, 0), half=(0.03, 0.03, 0.03), mass=0.216))
    return make_model(bodies, root_fixed=root_fixed, root_p=root_p)


def qdot_from_v(m, q, v):
    """Time derivative of the configuration for generalized velocity v."""
    q = np.asarray(q, float)
    v = np.asarray(v, float)
    if m.root_fixed:
        return v.copy()
    qd = np.zeros(O.nq(m))
    qd[0:3] = v[0:3]
    w, x, y, z = q[3:7]
    ox, oy, oz = v[3:6]
    # 1/2 quat (x) (0, omega_body)
    qd[3] = 0.5 * (-x * ox - y * oy - z * oz)
    qd[4] = 0.5 * (w * ox + y * oz - z * oy)
    qd[5] = 0.5 * (w * oy - x * oz + z * ox)
    qd[6] = 0.5 * (w * oz + x * oy - y * ox)
    qd[7:] = v[6:]
    return qd


def box_inertia_body(m, b):
    h = np.array(m.half[b][:])
    mb = m.mass[b]
    return mb / 3.0 * np.array([h[1] ** 2 + h[2] ** 2, h[0] ** 2 + h[2] ** 2, h[0] ** 2 + h[1] ** 2])


def body_rates_fd(m, q, v, eps=1e-6):
    """Per-body COM velocity and world angular velocity from FK differences."""
    qd = qdot_from_v(m, q, v)
    Rp, _, cp = O.fk(m, np.asarray(q) + eps * qd)
    Rm, _, cm = O.fk(m, np.asarray(q) - eps * qd)
    R0, _, c0 = O.fk(m, q)
    vc = (cp - cm) / (2 * eps)
    om = np.zeros((m.nb, 3))
    for b in range(m.nb):
        Rd = (Rp[b] - Rm[b]) / (2 * eps)
        W = Rd @ R0[b].T
        om[b] = [0.5 * (W[2, 1] - W[1, 2]), 0.5 * (W[0, 2] - W[2, 0]), 0.5 * (W[1, 0] - W[0, 1])]
    return vc, om, R0, c0


def kinetic_energy_fd(m, q, v):
    vc, om, R, _ = body_rates_fd(m, q, v)
    T = 0.0
    for b in range(m.nb):
        Iw = R[b] @ np.diag(box_inertia_body(m, b)) @ R[b].T
        T += 0.5 * m.mass[b] * vc[b] @ vc[b] + 0.5 * om[b] @ Iw @ om[b]
    return T


def momentum_fd(m, q, v):
    """Linear momentum and angular momentum about the world origin."""
    vc, om, R, c = body_rates_fd(m, q, v)
    P = np.zeros(3)
    Lo = np.zeros(3)
    for b in range(m.nb):
        Iw = R[b] @ np.diag(box_inertia_body(m, b)) @ R[b].T
        P += m.mass[b] * vc[b]
        Lo += np.cross(c[b], m.mass[b] * vc[b]) + Iw @ om[b]
    return P, Lo


def potential(m, q, g=9.81):
    _, _, c = O.fk(m, q)
    return sum(m.mass[b] * g * c[b][2] for b in range(m.nb))
