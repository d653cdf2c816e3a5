"""ctypes front end of the oracle's FP32 build (liborc32.so).

TEST INFRASTRUCTURE ONLY, like oracle.py.  The same C source as the FP64
oracle, compiled with its scalar type set to float (and single-precision
constants and library routines), so that every statement is evaluated in the
same order in FP32.  It answers one question for the parity tests: how far
from the FP64 oracle does FP32 arithmetic alone take one step of this method,
on a given state?  That spread is what any FP32 implementation of the method
carries, whatever its kernel does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import oracle as O

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc32.so")
F = C.c_float


class Model32(C.Structure):
    _fields_ = [
        ("nb", C.c_int32), ("root_fixed", C.c_int32),
        ("parent", C.c_int32 * O.MAXB), ("axis", C.c_int32 * O.MAXB),
        ("exclude", C.c_uint64 * O.MAXB),
        ("R_fix", (F * 9) * O.MAXB), ("p_fix", (F * 3) * O.MAXB),
        ("half", (F * 3) * O.MAXB), ("com", (F * 3) * O.MAXB),
        ("mass", F * O.MAXB), ("w_int", F * O.MAXB), ("w_cpl", F * O.MAXB),
        ("root_R", F * 9), ("root_p", F * 3),
        ("geom", C.c_int32 * O.MAXB),
    ]


class Params32(C.Structure):
    _fields_ = [
        ("dt", F), ("gravity", F * 3), ("pgs_iters", C.c_int32),
        ("soft_tau", F), ("soft_zeta", F), ("mu", F), ("contact_cap", C.c_int32),
        ("kp", F), ("kd", F), ("tau_max", F), ("theta_max", F), ("armature", F),
        ("ground", C.c_int32), ("box_box", C.c_int32), ("actuate", C.c_int32),
        ("max_correct_vel", F), ("min_cfm", F),
    ]


class ContactList32(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("a", C.c_int32 * O.MAXCAND), ("b", C.c_int32 * O.MAXCAND),
        ("p", (F * 3) * O.MAXCAND), ("nrm", (F * 3) * O.MAXCAND), ("depth", F * O.MAXCAND),
    ]


def contacts(m64: O.Model, q, prm: O.Params | None = None) -> dict:
    """Contact list of one configuration, evaluated in FP32."""
    m = Model32()
    _copy(m, m64)
    q = np.ascontiguousarray(q, dtype=np.float32)
    cl = ContactList32()
    mg = C.c_float(0.0)
    st = lib().orc_contacts(C.byref(m), C.byref(params32(prm or O.default_params())),
                            q.ctypes.data_as(C.POINTER(F)), C.byref(cl), C.byref(mg))
    n = cl.n
    return dict(a=np.array(cl.a[:n]), b=np.array(cl.b[:n]), depth=np.array(cl.depth[:n], np.float64),
                n=np.array([list(cl.nrm[k]) for k in range(n)]).reshape(n, 3),
                p=np.array([list(cl.p[k]) for k in range(n)]).reshape(n, 3), status=st, margin=mg.value)


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "orc.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "orc.h"))):
        subprocess.check_call(["make", "-s", "-C", _HERE, "-B", "liborc32.so"])
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.orc_run_many.argtypes = [P(Model32), C.c_int, P(Params32), C.c_int, P(F), C.c_int, P(F), C.c_int,
                                   P(F), C.c_int, P(C.c_uint32), P(O.Stats), C.c_int]
        L.orc_contacts.argtypes = [P(Model32), P(Params32), P(F), P(ContactList32), P(F)]
        _lib = L
    return _lib


def _copy(dst: C.Structure, src: C.Structure):
    """Field-by-field copy (FP64 values rounded to FP32)."""
    for name, _ in src._fields_:
        a = getattr(src, name)
        if isinstance(a, C.Array):
            b = getattr(dst, name)
            for i in range(len(a)):
                if isinstance(a[i], C.Array):
                    for j in range(len(a[i])):
                        b[i][j] = a[i][j]
                else:
                    b[i] = a[i]
        else:
            setattr(dst, name, a)


def params32(prm: O.Params) -> Params32:
    out = Params32()
    _copy(out, prm)
    return out


def run_population(pop, q, v, s, nsteps: int, prm: O.Params | None = None, threads: int = 1):
    """Every robot of ``pop`` ``nsteps`` steps in FP32; returns float64 copies
    of (q, v, s), the status words and the statistics."""
    prm = prm or O.default_params()
    models64 = O.models_from_population(pop)
    models = (Model32 * pop.n)()
    for i in range(pop.n):
        _copy(models[i], models64[i])
    q = np.ascontiguousarray(q, dtype=np.float32).copy()
    v = np.ascontiguousarray(v, dtype=np.float32).copy()
    s = np.ascontiguousarray(s, dtype=np.float32).copy()
    st = np.zeros(pop.n, np.uint32)
    stats = O.Stats()
    fp = lambda a: a.ctypes.data_as(C.POINTER(F))
    lib().orc_run_many(models, pop.n, C.byref(params32(prm)), int(nsteps), fp(q), q.shape[1], fp(v), v.shape[1],
                       fp(s), s.shape[1], st.ctypes.data_as(C.POINTER(C.c_uint32)), C.byref(stats), int(threads))
    return q.astype(np.float64), v.astype(np.float64), s.astype(np.float64), st, stats
