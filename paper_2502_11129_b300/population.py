"""Seeded synthetic populations of modular robots (input generation only).

This module builds the *inputs* of a simulation: robot morphologies, their
controller weights and their initial states.  It holds none of the
simulator's arithmetic (no kinematics, dynamics, contacts or integration):
morphologies are assembled on an integer millimetre lattice with signed
permutation matrices, which is exact and needs no floating point.  Both the
CUDA path and the FP64 oracle are fed from here, so they see bit-identical
inputs.

Workload shapes follow the paper's benchmark scenes (Sec. 4, "Simulation
Parameters": many independent *variants* of one scene) and the evolutionary
robotics setting of Revolve2 (Sec. 1): a core cube with hinge-jointed bricks,
driven by a CPG.

Populations:
  * ``boxes``      -- independent free 0.1 m / 1 kg cubes dropped on a plane
                       (the BOX-like scene).
  * ``quadrupeds`` -- core cube + 8 bricks in a fixed quadruped tree.
  * ``grammar``    -- random trees with 2..20 hinged bricks from a seeded
                       tree grammar, bricks on random free faces at random
                       90-degree rotations, no self-overlap; optionally some
                       modules are balls (sphere geometry).
  * ``box_and_ball`` -- a core cube with one hinged ball, dropped (the
                       BOX_AND_BALL-like scene).
  * ``rope``       -- a core cube trailing a chain of up to 63 bricks (the
                       ARM_WITH_ROPE-like long chain; beyond 25 links the
                       simulator steps it with a block per robot).

Body convention (shared reading of the model description):
  * body 0 is the core; its frame origin is the core centre.
  * a brick's frame origin is its hinge point, the centre of the parent face
    it is attached to; the brick's box centre is 30 mm along the brick's +x
    (the outward face normal); the hinge axis is the brick's y axis (index 1).
  * joint frame ``R_fix, p_fix``: the child frame at zero hinge angle,
    expressed in the parent frame.
  * ``exclude``: per-body bit mask of bodies it never collides with.  Every
    pair of boxes that touch (share a face, edge or corner) in the zero pose
    is excluded, which covers each parent-child pair; such pairs are built
    adjacent on purpose and their contacts would have near-zero Jacobians.
"""
from __future__ import annotations

import dataclasses
import numpy as np

MAXB = 32                 # padded body slots per robot (default)
MAXB_LONG = 64            # slots of populations with chains beyond 32 bodies
MAX_HINGES = 20
CORE_HALF_MM = 50
BRICK_HALF_MM = 30
DENSITY = 1000.0          # kg / m^3
GEOM_BOX, GEOM_SPHERE = 0, 1
START_CLEARANCE_MM = 5    # lowest vertex of a robot starts 5 mm above the plane

# faces of a box in its own frame: +x, -x, +y, -y, +z, -z
_FACE_NORMALS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                          [0, 0, 1], [0, 0, -1]], dtype=np.int64)
_FACE_U = np.array([[0, 1, 0], [0, 1, 0], [0, 0, 1], [0, 0, 1],
                    [1, 0, 0], [1, 0, 0]], dtype=np.int64)
_ATTACH_FACE = 1          # a brick is attached through its own -x face


def _face_frame(face: int) -> np.ndarray:
    """Signed permutation whose columns are (n, u, n x u) for a face."""
    n = _FACE_NORMALS[face]
    u = _FACE_U[face]
    return np.stack([n, u, np.cross(n, u)], axis=1)


def _rot_x_quarter(r: int) -> np.ndarray:
    """Rotation by r * 90 degrees about x, as an integer matrix."""
    c = [1, 0, -1, 0][r % 4]
    s = [0, 1, 0, -1][r % 4]
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.int64)


@dataclasses.dataclass
class Population:
    """Padded per-robot model description plus initial state.

    Arrays are indexed [robot, body] with ``slots`` body slots (MAXB, or
    MAXB_LONG for chains of more than 32 bodies).  Units are SI
    (metres, kilograms, radians).  Hinge i of a robot is body i+1.
    """
    kind: str
    n: int
    nb: np.ndarray            # (n,) int32 bodies per robot (1..21)
    parent: np.ndarray        # (n, MAXB) int8, -1 for the root / unused slots
    axis: np.ndarray          # (n, MAXB) int8 hinge axis index in child frame
    R_fix: np.ndarray         # (n, MAXB, 9) float64 row-major
    p_fix: np.ndarray         # (n, MAXB, 3) float64
    half: np.ndarray          # (n, MAXB, 3) float64 box half extents
    com: np.ndarray           # (n, MAXB, 3) float64 box centre in body frame
    mass: np.ndarray          # (n, MAXB) float64
    w_int: np.ndarray         # (n, MAXB) float64 CPG internal weight per hinge body
    w_cpl: np.ndarray         # (n, MAXB) float64 CPG coupling to the parent hinge
    q0: np.ndarray            # (n, MAXB+8) float64, first nq entries used
    v0: np.ndarray            # (n, MAXB+8) float64, first nv entries used
    exclude: np.ndarray       # (n, MAXB) uint64 bit j set: no contact with body j
    genome_face: np.ndarray   # (n, MAXB) int8 face of the parent each brick sits on
    genome_rot: np.ndarray    # (n, MAXB) int8 quarter-turn rotation of each brick
    geom: np.ndarray          # (n, MAXB) int8 GEOM_BOX, or GEOM_SPHERE (radius half[..., 0])

    @property
    def slots(self) -> int:
        return int(self.parent.shape[1])

    @property
    def nq(self) -> np.ndarray:
        return self.nb + 6

    @property
    def nv(self) -> np.ndarray:
        return self.nb + 5

    def subset(self, idx) -> "Population":
        idx = np.asarray(idx)
        fields = {}
        for f in dataclasses.fields(self):
            val = getattr(self, f.name)
            if isinstance(val, np.ndarray):
                fields[f.name] = val[idx].copy()
            else:
                fields[f.name] = val
        fields["n"] = int(len(idx))
        return Population(**fields)

    def as_float32(self) -> "Population":
        """Copy whose float fields are rounded to float32 (kept as float64)."""
        fields = {}
        for f in dataclasses.fields(self):
            val = getattr(self, f.name)
            if isinstance(val, np.ndarray) and val.dtype == np.float64:
                val = val.astype(np.float32).astype(np.float64)
            elif isinstance(val, np.ndarray):
                val = val.copy()
            fields[f.name] = val
        return Population(**fields)


def _empty(kind: str, n: int, slots: int = MAXB) -> Population:
    return Population(
        kind=kind, n=n,
        nb=np.zeros(n, np.int32),
        parent=np.full((n, slots), -1, np.int8),
        axis=np.zeros((n, slots), np.int8),
        R_fix=np.tile(np.eye(3).reshape(1, 1, 9), (n, slots, 1)),
        p_fix=np.zeros((n, slots, 3)),
        half=np.zeros((n, slots, 3)),
        com=np.zeros((n, slots, 3)),
        mass=np.zeros((n, slots)),
        w_int=np.zeros((n, slots)),
        w_cpl=np.zeros((n, slots)),
        q0=np.zeros((n, slots + 8)),
        v0=np.zeros((n, slots + 8)),
        exclude=np.zeros((n, slots), np.uint64),
        genome_face=np.full((n, slots), -1, np.int8),
        genome_rot=np.zeros((n, slots), np.int8),
        geom=np.zeros((n, slots), np.int8),
    )


def _box_mass(half_mm) -> float:
    side = 2.0 * np.asarray(half_mm, dtype=np.float64) / 1000.0
    return float(DENSITY * side[0] * side[1] * side[2])


def _ball_mass(radius_mm) -> float:
    r = float(radius_mm) / 1000.0
    return float(DENSITY * 4.0 / 3.0 * np.pi * r ** 3)


class _Lattice:
    """A robot under construction: exact zero-pose placement in millimetres."""

    def __init__(self):
        self.parent = [-1]
        self.face = [-1]
        self.rot = [0]
        self.R_world = [np.eye(3, dtype=np.int64)]           # body frame -> world
        self.origin = [np.zeros(3, np.int64)]                 # frame origin, world
        self.centre = [np.zeros(3, np.int64)]                 # box centre, world
        self.half = [np.array([CORE_HALF_MM] * 3, np.int64)]  # in body axes
        self.com_local = [np.zeros(3, np.int64)]
        self.R_fix = [np.eye(3, dtype=np.int64)]
        self.p_fix = [np.zeros(3, np.int64)]
        self.used_faces = [set()]
        self.geom = [GEOM_BOX]

    def free_faces(self, b: int):
        if self.geom[b] == GEOM_SPHERE:
            return []  # a ball module is a leaf
        faces = [f for f in range(6) if f not in self.used_faces[b]]
        if b > 0:
            faces = [f for f in faces if f != _ATTACH_FACE]
        return faces

    def propose(self, p: int, face: int, r: int):
        """Zero-pose placement of a brick on face ``face`` of body ``p``."""
        n = _FACE_NORMALS[face]
        ax = int(np.argmax(np.abs(n)))
        p_fix = self.com_local[p] + self.half[p][ax] * n
        R_fix = _face_frame(face) @ _rot_x_quarter(r)
        R_w = self.R_world[p] @ R_fix
        origin = self.origin[p] + self.R_world[p] @ p_fix
        com_local = np.array([BRICK_HALF_MM, 0, 0], np.int64)
        centre = origin + R_w @ com_local
        half = np.array([BRICK_HALF_MM] * 3, np.int64)
        return R_fix, p_fix, R_w, origin, centre, half, com_local

    def overlaps(self, centre, half_local, R_w) -> bool:
        ext = np.abs(R_w) @ half_local
        for c2, h2, R2 in zip(self.centre, self.half, self.R_world):
            e2 = np.abs(R2) @ h2
            # both boxes' axis-aligned extents shrunk by 1 mm
            if np.all(np.abs(centre - c2) < (ext - 1) + (e2 - 1)):
                return True
        return False

    def add(self, p, face, r, placed, geom=GEOM_BOX):
        """Attach a module; a ball (geom GEOM_SPHERE) fills the brick's cube
        (radius = the brick's half size) and its zero-pose overlap and touch
        tests use that cube, a conservative bound."""
        R_fix, p_fix, R_w, origin, centre, half, com_local = placed
        self.geom.append(geom)
        self.parent.append(p)
        self.face.append(face)
        self.rot.append(r)
        self.R_world.append(R_w)
        self.origin.append(origin)
        self.centre.append(centre)
        self.half.append(half)
        self.com_local.append(com_local)
        self.R_fix.append(R_fix)
        self.p_fix.append(p_fix)
        self.used_faces.append(set())
        self.used_faces[p].add(face)

    def touching_pairs(self):
        """Pairs of boxes whose closed extents touch or overlap at zero pose."""
        ext = [np.abs(R) @ h for R, h in zip(self.R_world, self.half)]
        out = []
        for a in range(len(self.centre)):
            for b in range(a + 1, len(self.centre)):
                if np.all(np.abs(self.centre[a] - self.centre[b]) <= ext[a] + ext[b]):
                    out.append((a, b))
        return out

    def lowest_vertex_mm(self) -> int:
        low = None
        for c, h, R, g in zip(self.centre, self.half, self.R_world, self.geom):
            z = int(c[2] - (h[0] if g == GEOM_SPHERE else (np.abs(R) @ h)[2]))
            low = z if low is None else min(low, z)
        return low


def _write_robot(pop: Population, i: int, lat: _Lattice, rng, quad_weights=None):
    nb = len(lat.parent)
    pop.nb[i] = nb
    for b in range(nb):
        pop.parent[i, b] = lat.parent[b]
        pop.axis[i, b] = 1 if b > 0 else 0
        pop.R_fix[i, b] = lat.R_fix[b].astype(np.float64).reshape(9)
        pop.p_fix[i, b] = lat.p_fix[b] / 1000.0
        pop.half[i, b] = lat.half[b] / 1000.0
        pop.com[i, b] = lat.com_local[b] / 1000.0
        pop.geom[i, b] = lat.geom[b]
        pop.mass[i, b] = _ball_mass(lat.half[b][0]) if lat.geom[b] == GEOM_SPHERE else _box_mass(lat.half[b])
        pop.genome_face[i, b] = lat.face[b]
        pop.genome_rot[i, b] = lat.rot[b]
    for a, b in lat.touching_pairs():
        pop.exclude[i, a] |= np.uint64(1 << b)
        pop.exclude[i, b] |= np.uint64(1 << a)
    w_int = rng.uniform(-1.0, 1.0, size=nb)
    w_cpl = rng.uniform(-1.0, 1.0, size=nb)
    for b in range(1, nb):
        pop.w_int[i, b] = w_int[b]
        pop.w_cpl[i, b] = w_cpl[b] if lat.parent[b] >= 1 else 0.0
    z0 = (START_CLEARANCE_MM - lat.lowest_vertex_mm()) / 1000.0
    pop.q0[i, :7] = [0.0, 0.0, z0, 1.0, 0.0, 0.0, 0.0]


def boxes(n: int, seed: int = 1, z_range=(0.2, 1.0), vel_sigma=0.5) -> Population:
    """Independent free cubes (0.1 m, 1 kg) above a plane.

    Height U[z_range], orientation a normalised N(0, I4) quaternion, linear and
    angular (body-frame) velocity components N(0, vel_sigma^2).
    """
    rng = np.random.default_rng(seed)
    pop = _empty("boxes", n)
    for i in range(n):
        lat = _Lattice()
        pop.nb[i] = 1
        pop.half[i, 0] = CORE_HALF_MM / 1000.0
        pop.mass[i, 0] = _box_mass(lat.half[0])
        z = rng.uniform(*z_range)
        quat = rng.normal(size=4)
        quat /= np.linalg.norm(quat)
        pop.q0[i, :7] = [0.0, 0.0, z, *quat]
        pop.v0[i, :6] = rng.normal(0.0, vel_sigma, size=6)
    return pop


def quadruped_lattice() -> _Lattice:
    lat = _Lattice()
    # hips on the core's side faces: hinge axis vertical
    for face, r in ((0, 1), (1, 1), (2, 0), (3, 0)):
        lat.add(0, face, r, lat.propose(0, face, r))
    # knees on each hip's outer face: hinge axis horizontal, across the leg
    for hip in range(1, 5):
        lat.add(hip, 0, 1, lat.propose(hip, 0, 1))
    return lat


def quadrupeds(n: int, seed: int = 2) -> Population:
    """Core cube + 4 hips + 4 knees; CPG weights U[-1, 1]."""
    rng = np.random.default_rng(seed)
    pop = _empty("quadrupeds", n)
    for i in range(n):
        _write_robot(pop, i, quadruped_lattice(), rng)
    return pop


def grammar_lattice(rng, n_hinges: int, max_tries: int = 100, ball_p: float = 0.0):
    """Random tree: each brick goes on a random free face of a random body;
    with probability ``ball_p`` a module is a ball (a leaf) instead."""
    while True:
        lat = _Lattice()
        ok = True
        for _ in range(n_hinges):
            placed = False
            for _try in range(max_tries):
                p = int(rng.integers(0, len(lat.parent)))
                faces = lat.free_faces(p)
                if not faces:
                    continue
                face = int(faces[rng.integers(0, len(faces))])
                r = int(rng.integers(0, 4))
                cand = lat.propose(p, face, r)
                if lat.overlaps(cand[4], cand[5], cand[2]):
                    continue
                geom = GEOM_BOX
                if ball_p > 0.0 and rng.uniform() < ball_p:
                    geom = GEOM_SPHERE
                lat.add(p, face, r, cand, geom)
                placed = True
                break
            if not placed:
                ok = False
                break
        if ok:
            return lat


def grammar(n: int, seed: int = 3, hinges=(2, MAX_HINGES), ball_p: float = 0.0) -> Population:
    """Seeded tree-grammar robots with U{hinges} hinged modules each; a module
    is a ball with probability ``ball_p`` (0: bricks only, the default)."""
    rng = np.random.default_rng(seed)
    pop = _empty("grammar" if ball_p == 0.0 else "grammar_balls", n)
    for i in range(n):
        nh = int(rng.integers(hinges[0], hinges[1] + 1))
        _write_robot(pop, i, grammar_lattice(rng, nh, ball_p=ball_p), rng)
    return pop


def box_and_ball(n: int, seed: int = 4, z_range=(0.1, 0.5), vel_sigma=0.5) -> Population:
    """A core cube with one ball module on a random face, hinged, dropped like
    ``boxes``: height U[z_range] added to the resting clearance, orientation a
    normalised N(0, I4) quaternion, root velocity components N(0, vel_sigma^2).
    Sphere/plane and box/plane contacts (the ball and the core are adjacent
    and never collide with each other)."""
    rng = np.random.default_rng(seed)
    pop = _empty("box_and_ball", n)
    for i in range(n):
        lat = _Lattice()
        face = int(rng.integers(0, 6))
        r = int(rng.integers(0, 4))
        lat.add(0, face, r, lat.propose(0, face, r), GEOM_SPHERE)
        _write_robot(pop, i, lat, rng)
        quat = rng.normal(size=4)
        quat /= np.linalg.norm(quat)
        # clear of the plane in any orientation: the robot's bounding radius
        reach = (CORE_HALF_MM * np.sqrt(3.0) + 2 * BRICK_HALF_MM + CORE_HALF_MM) / 1000.0
        pop.q0[i, :7] = [0.0, 0.0, reach + rng.uniform(*z_range), *quat]
        pop.v0[i, :6] = rng.normal(0.0, vel_sigma, size=6)
    return pop


def rope_lattice(links: int) -> _Lattice:
    """Core cube with a straight chain of ``links`` bricks on its +x face,
    each on the +x face of the one before, hinge axes alternating between
    the bricks' y and z (quarter turn every second link)."""
    lat = _Lattice()
    p = 0
    for k in range(links):
        r = k % 2
        lat.add(p, 0, r, lat.propose(p, 0, r))
        p = len(lat.parent) - 1
    return lat


def rope(n: int, seed: int = 5, links: int = 25) -> Population:
    """A long chain (up to 63 links, the per-robot body bound of 64): a core
    cube trailing a chain of bricks, dropped from U[0, 0.3] m above its
    resting height, bent in the horizontal plane (vertical-axis hinges
    U[-0.3, 0.3], the others straight), hinge rates N(0, 1).  Run with
    actuate=0 the chain is passive (a rope); with the CPG on it is a snake.
    Chains of more than 25 links (more than 31 dofs) take the simulator's
    block-per-robot path; more than 31 links need MAXB_LONG body slots."""
    if not 1 <= links <= MAXB_LONG - 1:
        raise ValueError(f"links must be in 1..{MAXB_LONG - 1}")
    rng = np.random.default_rng(seed)
    pop = _empty("rope", n, MAXB if links + 1 <= MAXB else MAXB_LONG)
    lat = rope_lattice(links)
    vertical = np.array([k % 2 == 1 for k in range(links)])  # quarter-turned links
    for i in range(n):
        _write_robot(pop, i, lat, rng)
        pop.q0[i, 2] += rng.uniform(0.0, 0.3)
        pop.q0[i, 7:7 + links] = np.where(vertical, rng.uniform(-0.3, 0.3, size=links), 0.0)
        pop.v0[i, 6:6 + links] = rng.normal(0.0, 1.0, size=links)
    return pop


def concat(pops) -> Population:
    """One population of several (kind of the first): body-slot arrays are
    padded to the largest slot count (unused slots as _empty leaves them)."""
    pops = list(pops)
    slots = max(p.slots for p in pops)
    pad_value = {"parent": -1, "genome_face": -1}
    fields = {}
    for f in dataclasses.fields(Population):
        vals = [getattr(p, f.name) for p in pops]
        if not isinstance(vals[0], np.ndarray):
            fields[f.name] = vals[0]
            continue
        if f.name == "nb":
            fields[f.name] = np.concatenate(vals)
            continue
        out = []
        for p, x in zip(pops, vals):
            extra = slots - p.slots
            if extra:
                widths = [(0, 0)] * x.ndim
                widths[1] = (0, extra)
                if f.name == "R_fix":
                    eye = np.tile(np.eye(3).reshape(1, 1, 9), (x.shape[0], extra, 1))
                    x = np.concatenate([x, eye], axis=1)
                else:
                    x = np.pad(x, widths, constant_values=pad_value.get(f.name, 0))
            out.append(x)
        fields[f.name] = np.concatenate(out)
    fields["n"] = int(sum(p.n for p in pops))
    return Population(**fields)


def lift(pop: Population, dz: float) -> Population:
    """Copy of ``pop`` with every root raised by ``dz`` metres."""
    out = pop.subset(np.arange(pop.n))
    out.q0[:, 2] += dz
    return out


def random_state(pop: Population, seed: int, angle=0.6, rate=1.0, lin=0.5, ang=0.5):
    """Seeded random (q, v, cpg) for one-step parity tests.

    Hinge angles U[-angle, angle], hinge rates N(0, rate^2), root velocity
    components N(0, lin^2) / N(0, ang^2), orientation a normalised N(0, I4)
    quaternion.  CPG state N(0, 0.5^2).
    """
    rng = np.random.default_rng(seed)
    q = pop.q0.copy()
    v = np.zeros_like(pop.v0)
    s = np.zeros((pop.n, 2 * (pop.slots - 1)))
    for i in range(pop.n):
        nb = int(pop.nb[i])
        quat = rng.normal(size=4)
        quat /= np.linalg.norm(quat)
        q[i, 3:7] = quat
        q[i, 7:7 + nb - 1] = rng.uniform(-angle, angle, size=nb - 1)
        v[i, 0:3] = rng.normal(0.0, lin, size=3)
        v[i, 3:6] = rng.normal(0.0, ang, size=3)
        v[i, 6:6 + nb - 1] = rng.normal(0.0, rate, size=nb - 1)
        s[i, : 2 * (nb - 1)] = rng.normal(0.0, 0.5, size=2 * (nb - 1))
    return q, v, s


def cpg_initial(pop: Population) -> np.ndarray:
    """Initial oscillator state: x = y = 1/sqrt(2) for every hinge."""
    s = np.zeros((pop.n, 2 * (pop.slots - 1)))
    for i in range(pop.n):
        nh = int(pop.nb[i]) - 1
        s[i, : 2 * nh] = np.sqrt(0.5)
    return s
