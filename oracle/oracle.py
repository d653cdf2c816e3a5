"""ctypes front end of the FP64 oracle (oracle/orc.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this module.  It shares no code
with the CUDA path; both are fed by ``paper_2502_11129_b300.population``.

What pins each oracle function (tests/test_oracle_pins.py):
  * integrate + gravity     -- free-fall exact discrete closed form; projectile.
  * FK                      -- hand-computed poses of a two-brick chain.
  * CRBA mass matrix        -- brute force from kinetic energy evaluated with
                               finite differences of FK positions/rotations.
  * RNEA bias               -- Lagrange's equations by finite differences of M
                               (fixed-root chains); momentum balance of free
                               robots (rate of linear/angular momentum equals
                               the gravity wrench).
  * Cholesky / solves       -- residual and an independent LU solve.
  * hinge dynamics          -- small-angle compound-pendulum period; energy
                               drift of a chain shrinking linearly with dt.
  * torque-free rotation    -- isotropic cube: body rate and world angular
                               momentum exactly constant.
  * contacts                -- hand-placed boxes (vertex depths, face-face
                               four-point patch, crossed-edge point).
  * soft PGS                -- single-contact closed form after one sweep;
                               resting cube steady penetration closed form;
                               incline stick/slide threshold tan(a) = mu.
  * CPG                     -- norm growth sqrt(1 + dt^2 w^2)^n of one
                               oscillator.
  * fitness                 -- xy displacement of a translated body.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")

MAXB = 64
MAXV = 70
MAXQ = 71
MAXCAND = 4096
NPHASE = 9
PHASES = ["cpg", "fk", "rnea", "crba", "chol", "contact", "jac", "pgs", "integ"]
ST_NONFINITE, ST_OVERFLOW, ST_CHOL = 1, 2, 4


class Model(C.Structure):
    _fields_ = [
        ("nb", C.c_int32), ("root_fixed", C.c_int32),
        ("parent", C.c_int32 * MAXB), ("axis", C.c_int32 * MAXB),
        ("exclude", C.c_uint64 * MAXB),
        ("R_fix", (C.c_double * 9) * MAXB), ("p_fix", (C.c_double * 3) * MAXB),
        ("half", (C.c_double * 3) * MAXB), ("com", (C.c_double * 3) * MAXB),
        ("mass", C.c_double * MAXB), ("w_int", C.c_double * MAXB),
        ("w_cpl", C.c_double * MAXB),
        ("root_R", C.c_double * 9), ("root_p", C.c_double * 3),
        ("geom", C.c_int32 * MAXB),
    ]


class Params(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("pgs_iters", C.c_int32),
        ("soft_tau", C.c_double), ("soft_zeta", C.c_double), ("mu", C.c_double),
        ("contact_cap", C.c_int32),
        ("kp", C.c_double), ("kd", C.c_double), ("tau_max", C.c_double),
        ("theta_max", C.c_double), ("armature", C.c_double),
        ("ground", C.c_int32), ("box_box", C.c_int32), ("actuate", C.c_int32),
        ("max_correct_vel", C.c_double), ("min_cfm", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("flops", C.c_double * NPHASE), ("contacts", C.c_double),
        ("narrow_pairs", C.c_double), ("broad_pairs", C.c_double),
        ("margin", C.c_double), ("overflow_steps", C.c_int32), ("steps", C.c_int32),
    ]


class ContactList(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("a", C.c_int32 * MAXCAND), ("b", C.c_int32 * MAXCAND),
        ("p", (C.c_double * 3) * MAXCAND), ("nrm", (C.c_double * 3) * MAXCAND),
        ("depth", C.c_double * MAXCAND),
    ]


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (plain C, FP64)."""
    src = os.path.join(_HERE, "orc.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "orc.h"))):
        subprocess.check_call(["make", "-s", "-C", _HERE, "-B", "liborc.so"])
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.orc_default_params.argtypes = [P(Params)]
        L.orc_fk.argtypes = [P(Model), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.orc_mass_matrix.argtypes = [P(Model), P(Params), P(C.c_double), P(C.c_double)]
        L.orc_bias.argtypes = [P(Model), P(Params), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.orc_cholesky.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
        L.orc_contacts.argtypes = [P(Model), P(Params), P(C.c_double), P(ContactList), P(C.c_double)]
        L.orc_step_detail.argtypes = [P(Model), P(Params), P(C.c_double), P(C.c_double),
                                      P(C.c_double), P(C.c_uint32), P(C.c_double),
                                      P(C.c_double), P(C.c_int32)]
        L.orc_run.argtypes = [P(Model), P(Params), C.c_int, P(C.c_double), P(C.c_double),
                              P(C.c_double), P(C.c_uint32), P(Stats)]
        L.orc_contacts_flip.argtypes = [P(Model), P(Params), P(C.c_double), C.c_double, P(C.c_int32), C.c_int32,
                                        P(ContactList), P(C.c_int32), P(C.c_int32), P(C.c_double)]
        L.orc_step_flip.argtypes = [P(Model), P(Params), P(C.c_double), P(C.c_double), P(C.c_double),
                                    P(C.c_uint32), C.c_double, P(C.c_int32), C.c_int32, P(C.c_int32),
                                    P(C.c_int32), P(C.c_double)]
        L.orc_run_many.argtypes = [P(Model), C.c_int, P(Params), C.c_int, P(C.c_double), C.c_int,
                                   P(C.c_double), C.c_int, P(C.c_double), C.c_int,
                                   P(C.c_uint32), P(Stats), C.c_int]
        assert L.orc_sizeof_model() == C.sizeof(Model)
        assert L.orc_sizeof_params() == C.sizeof(Params)
        assert L.orc_sizeof_stats() == C.sizeof(Stats)
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "gravity":
            for i in range(3):
                p.gravity[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def model_from_population(pop, i: int) -> Model:
    """orc_model of robot ``i`` of a population (float64 values as stored)."""
    m = Model()
    nb = int(pop.nb[i])
    m.nb = nb
    m.root_fixed = 0
    for b in range(min(MAXB, pop.parent.shape[1])):
        m.parent[b] = int(pop.parent[i, b])
        m.axis[b] = int(pop.axis[i, b])
        m.exclude[b] = int(pop.exclude[i, b])
        for k in range(9):
            m.R_fix[b][k] = float(pop.R_fix[i, b, k])
        for k in range(3):
            m.p_fix[b][k] = float(pop.p_fix[i, b, k])
            m.half[b][k] = float(pop.half[i, b, k])
            m.com[b][k] = float(pop.com[i, b, k])
        m.mass[b] = float(pop.mass[i, b])
        m.w_int[b] = float(pop.w_int[i, b])
        m.w_cpl[b] = float(pop.w_cpl[i, b])
        m.geom[b] = int(pop.geom[i, b])
    for k in range(9):
        m.root_R[k] = 1.0 if k in (0, 4, 8) else 0.0
    return m


def models_from_population(pop):
    arr = (Model * pop.n)()
    for i in range(pop.n):
        arr[i] = model_from_population(pop, i)
    return arr


def nq(m: Model) -> int:
    return (0 if m.root_fixed else 7) + m.nb - 1


def nv(m: Model) -> int:
    return (0 if m.root_fixed else 6) + m.nb - 1


def fk(m: Model, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros((m.nb, 9)); p = np.zeros((m.nb, 3)); c = np.zeros((m.nb, 3))
    lib().orc_fk(C.byref(m), _dp(q), _dp(R), _dp(p), _dp(c))
    return R.reshape(m.nb, 3, 3), p, c


def mass_matrix(m: Model, q, prm: Params | None = None):
    prm = prm or default_params()
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = nv(m)
    M = np.zeros((n, n))
    lib().orc_mass_matrix(C.byref(m), C.byref(prm), _dp(q), _dp(M))
    return M


def bias(m: Model, q, v, prm: Params | None = None):
    prm = prm or default_params()
    q = np.ascontiguousarray(q, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    c = np.zeros(nv(m))
    lib().orc_bias(C.byref(m), C.byref(prm), _dp(q), _dp(v), _dp(c))
    return c


def cholesky(M):
    M = np.ascontiguousarray(M, dtype=np.float64)
    L = np.zeros_like(M)
    rc = lib().orc_cholesky(M.shape[0], _dp(M), _dp(L))
    return rc, L


def contacts(m: Model, q, prm: Params | None = None):
    prm = prm or default_params()
    q = np.ascontiguousarray(q, dtype=np.float64)
    cl = ContactList()
    margin = C.c_double(0.0)
    st = lib().orc_contacts(C.byref(m), C.byref(prm), _dp(q), C.byref(cl), C.byref(margin))
    n = cl.n
    out = dict(
        a=np.array(cl.a[:n]), b=np.array(cl.b[:n]),
        p=np.array([list(cl.p[k]) for k in range(n)]).reshape(n, 3),
        n=np.array([list(cl.nrm[k]) for k in range(n)]).reshape(n, 3),
        depth=np.array(cl.depth[:n]), status=st, margin=margin.value,
    )
    return out


def step_detail(m: Model, q, v, s, prm: Params | None = None, status: int = 0):
    prm = prm or default_params()
    q = np.array(q, dtype=np.float64); v = np.array(v, dtype=np.float64)
    s = np.array(s, dtype=np.float64)
    st = C.c_uint32(status)
    vfree = np.zeros(MAXV)
    lam = np.zeros(3 * 256)
    nc = C.c_int32(0)
    lib().orc_step_detail(C.byref(m), C.byref(prm), _dp(q), _dp(v), _dp(s), C.byref(st),
                          _dp(vfree), _dp(lam), C.byref(nc))
    return dict(q=q, v=v, s=s, status=st.value, vfree=vfree[:nv(m)],
                lam=lam[:3 * nc.value].reshape(-1, 3), nc=nc.value)


def run(m: Model, q, v, s, nsteps: int, prm: Params | None = None, status: int = 0):
    """Run one variant ``nsteps`` steps; returns (q, v, s, status, stats)."""
    prm = prm or default_params()
    q = np.array(q, dtype=np.float64); v = np.array(v, dtype=np.float64)
    s = np.array(s, dtype=np.float64)
    if s.size == 0:
        s = np.zeros(2 * MAXB)
    st = C.c_uint32(status)
    stats = Stats()
    lib().orc_run(C.byref(m), C.byref(prm), int(nsteps), _dp(q), _dp(v), _dp(s),
                  C.byref(st), C.byref(stats))
    return q, v, s, st.value, stats


MAXNEAR = 64


def step_flip(m: Model, q, v, s, flips=(), band: float = 1e-5, prm: Params | None = None, status: int = 0):
    """One step with the near-threshold decisions numbered in ``flips`` taken
    the other way (orc_step_flip).  Returns (q, v, s, status, near, margin):
    ``near`` are the numbers of the decisions within ``band`` that the step
    met (at most MAXNEAR listed)."""
    prm = prm or default_params()
    q = np.array(q, dtype=np.float64); v = np.array(v, dtype=np.float64)
    s = np.array(s, dtype=np.float64)
    if s.size == 0:
        s = np.zeros(2 * MAXB)
    st = C.c_uint32(status)
    fl = np.ascontiguousarray(list(flips), dtype=np.int32)
    near = np.zeros(MAXNEAR, np.int32)
    nn = C.c_int32(0)
    mg = C.c_double(0.0)
    rc = lib().orc_step_flip(C.byref(m), C.byref(prm), _dp(q), _dp(v), _dp(s), C.byref(st), float(band),
                             fl.ctypes.data_as(C.POINTER(C.c_int32)) if fl.size else None, int(fl.size),
                             near.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nn), C.byref(mg))
    if rc != 0:
        raise ValueError("orc_step_flip: bad arguments")
    return q, v, s, st.value, near[:min(nn.value, MAXNEAR)].copy(), mg.value


def _contact_dict(cl, st, margin):
    n = cl.n
    return dict(a=np.array(cl.a[:n]), b=np.array(cl.b[:n]),
                p=np.array([list(cl.p[k]) for k in range(n)]).reshape(n, 3),
                n=np.array([list(cl.nrm[k]) for k in range(n)]).reshape(n, 3),
                depth=np.array(cl.depth[:n]), status=st, margin=margin)


def contact_outcomes(m: Model, q, band: float = 1e-5, prm: Params | None = None, max_runs: int = 512):
    """Every valid contact list of one configuration: the tree of its
    decisions within ``band`` of their thresholds (as step_outcomes).
    Returns (lists, n_near, complete); lists[0] is the plain one."""
    prm = prm or default_params()
    q = np.ascontiguousarray(q, dtype=np.float64)
    outs = []
    stack = [()]
    n_near = 0
    while stack:
        if len(outs) >= max_runs:
            return outs, n_near, False
        S = stack.pop()
        cl = ContactList()
        fl = np.ascontiguousarray(S, dtype=np.int32)
        near = np.zeros(MAXNEAR, np.int32)
        nn = C.c_int32(0)
        mg = C.c_double(0.0)
        st = lib().orc_contacts_flip(C.byref(m), C.byref(prm), _dp(q), float(band),
                                     fl.ctypes.data_as(C.POINTER(C.c_int32)) if fl.size else None, int(fl.size),
                                     C.byref(cl), near.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nn),
                                     C.byref(mg))
        if st < 0:
            raise ValueError("orc_contacts_flip: bad arguments")
        if not S:
            n_near = min(nn.value, MAXNEAR)
        outs.append(_contact_dict(cl, st, mg.value))
        last = S[-1] if S else -1
        for x in sorted((int(x) for x in near[:min(nn.value, MAXNEAR)] if x > last), reverse=True):
            stack.append(S + (x,))
    return outs, n_near, True


def step_outcomes(m: Model, q, v, s, band: float = 1e-5, prm: Params | None = None, max_runs: int = 512):
    """Every valid outcome of one step whose discrete decisions may go either
    way: the tree of the step's decisions within ``band`` of their
    thresholds, explored depth first.  A run that reverses the decisions S
    reports the near decisions it meets, numbered in its own order; those
    numbered above max(S) sit after every reversed decision, so their numbers
    mean the same in the run reversing S + (x,), and every combination is
    reached once.  Returns (outcomes, n_near, complete): outcomes is a list of
    (q, v, s, status), the plain step first; n_near the plain step's near
    decisions; complete False if max_runs cut the tree."""
    outs = []
    stack = [()]
    n_near = 0
    while stack:
        if len(outs) >= max_runs:
            return outs, n_near, False
        S = stack.pop()
        qa, va, sa, sta, near, _ = step_flip(m, q, v, s, S, band, prm)
        if not S:
            n_near = len(near)
        outs.append((qa, va, sa, sta))
        last = S[-1] if S else -1
        for x in sorted((int(x) for x in near if x > last), reverse=True):
            stack.append(S + (x,))
    return outs, n_near, True


def run_population(pop, q, v, s, nsteps: int, prm: Params | None = None, threads: int = 1,
                   status=None, models=None):
    """Run every robot of ``pop`` ``nsteps`` steps with ``threads`` pthreads.

    q, v, s: (n, width) float64 arrays updated in place-copy and returned.
    """
    prm = prm or default_params()
    models = models if models is not None else models_from_population(pop)
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    s = np.ascontiguousarray(s, dtype=np.float64).copy()
    st = np.zeros(pop.n, np.uint32) if status is None else np.array(status, np.uint32)
    stats = Stats()
    lib().orc_run_many(models, pop.n, C.byref(prm), int(nsteps), _dp(q), q.shape[1], _dp(v),
                       v.shape[1], _dp(s), s.shape[1],
                       st.ctypes.data_as(C.POINTER(C.c_uint32)), C.byref(stats), int(threads))
    return q, v, s, st, stats


def stats_dict(st: Stats) -> dict:
    d = {f"flops_{p}": st.flops[i] for i, p in enumerate(PHASES)}
    d["flops_total"] = float(sum(st.flops[i] for i in range(NPHASE)))
    d.update(contacts=st.contacts, narrow_pairs=st.narrow_pairs, broad_pairs=st.broad_pairs,
             margin=st.margin, overflow_steps=st.overflow_steps, steps=st.steps)
    return d


def fitness(q_start, q_end) -> np.ndarray:
    """Core xy displacement between two configurations (free roots)."""
    q_start = np.atleast_2d(q_start); q_end = np.atleast_2d(q_end)
    return np.hypot(q_end[:, 0] - q_start[:, 0], q_end[:, 1] - q_start[:, 1])
