"""ctypes binding of libb3cpu (include/b3cpu.h): the host engine of the
population simulator, the CPU side of the paper's hybrid allocation (Sec. 6).

Argument marshalling only; every step runs in the library's C++ worker
threads.  The GPU simulator (sim.py) never calls this module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import population as popmod
from . import sim as S

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libb3cpu.so")
EXPORTS = ["cpu_create", "cpu_destroy", "cpu_set_population", "cpu_set_state", "cpu_step_n", "cpu_read_state",
           "cpu_fitness", "cpu_robot_seconds", "cpu_threads", "cpu_contacts", "cpu_last_error"]

_lib = None


def lib():
    """Load libb3cpu.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise S.SimError(f"{LIB_PATH} is missing; build it with python -m paper_2502_11129_b300.build")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.cpu_create.argtypes = [C.POINTER(S.SimConfig), C.c_int32, C.POINTER(vp)]
        L.cpu_destroy.argtypes = [vp]
        L.cpu_set_population.argtypes = [vp, C.POINTER(S.VariantDesc), C.c_int32]
        L.cpu_set_state.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.cpu_step_n.argtypes = [vp, C.c_int32]
        L.cpu_read_state.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp]
        L.cpu_fitness.argtypes = [vp, vp, C.c_int32]
        L.cpu_contacts.argtypes = [vp, C.POINTER(C.c_double)]
        L.cpu_robot_seconds.argtypes = [vp, vp, C.c_int32]
        L.cpu_threads.argtypes = [vp]
        L.cpu_last_error.argtypes = [vp]
        L.cpu_last_error.restype = C.c_char_p
        _lib = L
    return _lib


class CpuSim:
    """One host-engine context (same state layout and calls as sim.Sim)."""

    def __init__(self, threads: int = 0, **cfg):
        c = dict(S.DEFAULTS)
        c.update(cfg)
        self.cfg = c
        sc = S.SimConfig()
        for k, val in c.items():
            if k == "gravity":
                for i in range(3):
                    sc.gravity[i] = val[i]
            else:
                setattr(sc, k, val)
        h = C.c_void_p()
        rc = lib().cpu_create(C.byref(sc), int(threads), C.byref(h))
        if rc != 0:
            raise S.SimError(f"cpu_create: {S.STATUS.get(rc, rc)}")
        self.h = h
        self.n = 0

    def _check(self, rc, what):
        if rc != 0:
            raise S.SimError(f"{what}: {S.STATUS.get(rc, rc)}: {lib().cpu_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib().cpu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_population(self, pop: popmod.Population):
        p32 = S.Population32(pop)
        self._check(lib().cpu_set_population(self.h, p32.descs, pop.n), "cpu_set_population")
        self.n = pop.n

    def set_state(self, Q, V, Sx=None, first: int = 0):
        Q = np.ascontiguousarray(Q, np.float32)
        V = np.ascontiguousarray(V, np.float32)
        Sx = None if Sx is None else np.ascontiguousarray(Sx, np.float32)
        self._check(lib().cpu_set_state(self.h, first, Q.shape[0], S._ptr(Q), S._ptr(V), S._ptr(Sx)),
                    "cpu_set_state")

    def step(self, n_steps: int):
        self._check(lib().cpu_step_n(self.h, int(n_steps)), "cpu_step_n")

    def read_state(self, first: int = 0, count: int | None = None):
        count = self.n - first if count is None else count
        Q = np.zeros((count, S.SIM_QW), np.float32)
        V = np.zeros((count, S.SIM_VW), np.float32)
        Sx = np.zeros((count, S.SIM_SW), np.float32)
        st = np.zeros(count, np.uint32)
        self._check(lib().cpu_read_state(self.h, first, count, S._ptr(Q), S._ptr(V), S._ptr(Sx), S._ptr(st)),
                    "cpu_read_state")
        return Q, V, Sx, st

    def fitness(self, n: int | None = None):
        n = self.n if n is None else n
        out = np.zeros(n, np.float32)
        self._check(lib().cpu_fitness(self.h, S._ptr(out), n), "cpu_fitness")
        return out

    def robot_seconds(self):
        """Wall seconds of every robot in the last step call (caller order)."""
        out = np.zeros(self.n, np.float64)
        self._check(lib().cpu_robot_seconds(self.h, S._ptr(out), self.n), "cpu_robot_seconds")
        return out

    @property
    def threads(self) -> int:
        return int(lib().cpu_threads(self.h))

    def contacts(self) -> float:
        c = C.c_double()
        self._check(lib().cpu_contacts(self.h, C.byref(c)), "cpu_contacts")
        return c.value
