"""Python binding of the C ABI in include/b3sim.h (argument marshalling only).

Every step of the simulation runs in the CUDA library ``libb3sim.so``; this
module only converts numpy arrays to the ABI's structs and pointers.  There
is no CPU fallback: if the library is missing or no CUDA device is present,
construction raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import population as popmod

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libb3sim.so")

SIM_MAX_BODIES = 64
SIM_WARP_MAX_BODIES = 26
SIM_QW, SIM_VW, SIM_SW = 72, 72, 128
SIM_MAX_CONTACT_CAP = 64
ST_NONFINITE, ST_OVERFLOW, ST_CHOL, ST_CANDIDATES = 1, 2, 4, 8
STATUS = {0: "SIM_OK", -1: "SIM_EINVAL", -2: "SIM_ECUDA", -3: "SIM_ENOMEM", -4: "SIM_ESTATE"}

EXPORTS = ["sim_create", "sim_destroy", "sim_set_population", "sim_set_state", "sim_step_n",
           "sim_read_state", "sim_fitness", "sim_autotune", "sim_counters_read",
           "sim_debug_contacts", "sim_debug_solver", "sim_debug_sincos", "sim_robot_cost", "sim_launch_shape", "sim_step_n_noalloc", "sim_set_state_dev", "sim_read_state_dev",
           "sim_fitness_dev", "sim_stream", "sim_fp32_peak", "sim_last_error"]


class SimConfig(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("gravity", C.c_float * 3), ("pgs_iters", C.c_int32),
        ("soft_tau", C.c_float), ("soft_zeta", C.c_float), ("mu", C.c_float),
        ("contact_cap", C.c_int32), ("kp", C.c_float), ("kd", C.c_float),
        ("tau_max", C.c_float), ("theta_max", C.c_float), ("armature", C.c_float),
        ("ground", C.c_int32), ("box_box", C.c_int32), ("actuate", C.c_int32),
        ("max_correct_vel", C.c_float), ("device", C.c_int32), ("stream", C.c_uint64), ("steps_per_launch", C.c_int32),
        ("warps_per_block", C.c_int32), ("min_cfm", C.c_float), ("phase_lock", C.c_int32),
        ("warps_per_sm", C.c_int32),
    ]


class VariantDesc(C.Structure):
    _fields_ = [
        ("n_bodies", C.c_int32), ("parent", C.POINTER(C.c_int8)), ("hinge_axis", C.POINTER(C.c_int8)),
        ("exclude", C.POINTER(C.c_uint64)), ("joint_frame", C.POINTER(C.c_float)),
        ("half_size", C.POINTER(C.c_float)), ("box_center", C.POINTER(C.c_float)),
        ("mass", C.POINTER(C.c_float)), ("cpg_w_internal", C.POINTER(C.c_float)),
        ("cpg_w_couple", C.POINTER(C.c_float)), ("geom", C.POINTER(C.c_int8)),
    ]


class DevicePopulation(C.Structure):
    """Caller-owned device buffers for sim_step_n_noalloc (see b3sim.h)."""
    _fields_ = [("n", C.c_int32), ("model_f", C.c_void_p), ("model_i", C.c_void_p),
                ("meta", C.c_void_p), ("pairs", C.c_void_p), ("q", C.c_void_p), ("v", C.c_void_p),
                ("cpg", C.c_void_p), ("status", C.c_void_p)]


class Counters(C.Structure):
    _fields_ = [("contacts", C.c_double), ("narrow_pairs", C.c_double),
                ("broad_pairs", C.c_double), ("variant_steps", C.c_double), ("sm_cycles", C.c_double)]


DEFAULTS = dict(dt=0.002, gravity=(0.0, 0.0, -9.81), pgs_iters=30, soft_tau=0.02, soft_zeta=1.0,
                mu=1.0, contact_cap=64, kp=2.0, kd=0.05, tau_max=1.0, theta_max=np.pi / 2,
                armature=1e-4, ground=1, box_box=1, actuate=1, max_correct_vel=0.1, device=0, stream=0,
                steps_per_launch=0, warps_per_block=0, min_cfm=0.1, phase_lock=0, warps_per_sm=0)

_lib = None


class SimError(RuntimeError):
    pass


def lib():
    """Load libb3sim.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SimError(f"{LIB_PATH} is missing; build it with python -m paper_2502_11129_b300.build")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        vp = C.c_void_p
        L.sim_create.argtypes = [P(SimConfig), P(vp)]
        L.sim_destroy.argtypes = [vp]
        L.sim_set_population.argtypes = [vp, P(VariantDesc), C.c_int32]
        L.sim_set_state.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.sim_step_n.argtypes = [vp, C.c_int32]
        L.sim_read_state.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp]
        L.sim_fitness.argtypes = [vp, vp, C.c_int32]
        L.sim_autotune.argtypes = [vp, C.c_int32]
        L.sim_counters_read.argtypes = [vp, P(Counters)]
        L.sim_debug_contacts.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, P(C.c_int32)]
        L.sim_debug_solver.argtypes = [vp, C.c_int32, vp, vp, P(C.c_int32), vp]
        L.sim_step_n_noalloc.argtypes = [P(SimConfig), P(DevicePopulation), C.c_int32]
        L.sim_debug_sincos.argtypes = [vp, C.c_int32, vp, vp]
        L.sim_robot_cost.argtypes = [vp, vp, C.c_int32]
        L.sim_launch_shape.argtypes = [vp, vp, vp, vp, vp]
        L.sim_set_state_dev.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.sim_read_state_dev.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp]
        L.sim_fitness_dev.argtypes = [vp, vp, C.c_int32]
        L.sim_stream.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.sim_fp32_peak.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_float),
                                    C.POINTER(C.c_int32)]
        L.sim_last_error.argtypes = [vp]
        L.sim_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Population32:
    """float32 / int8 host copies of a Population laid out for the ABI."""

    def __init__(self, pop: popmod.Population):
        n = pop.n
        self.n = n
        self.parent = np.ascontiguousarray(pop.parent, dtype=np.int8)
        self.axis = np.ascontiguousarray(pop.axis, dtype=np.int8)
        self.exclude = np.ascontiguousarray(pop.exclude, dtype=np.uint64)
        jf = np.concatenate([pop.R_fix, pop.p_fix], axis=2)
        self.joint_frame = np.ascontiguousarray(jf, dtype=np.float32)
        self.half = np.ascontiguousarray(pop.half, dtype=np.float32)
        self.com = np.ascontiguousarray(pop.com, dtype=np.float32)
        self.mass = np.ascontiguousarray(pop.mass, dtype=np.float32)
        self.w_int = np.ascontiguousarray(pop.w_int, dtype=np.float32)
        self.w_cpl = np.ascontiguousarray(pop.w_cpl, dtype=np.float32)
        self.geom = np.ascontiguousarray(pop.geom, dtype=np.int8)
        self.descs = (VariantDesc * n)()
        f = C.POINTER(C.c_float)
        for i in range(n):
            d = self.descs[i]
            d.n_bodies = int(pop.nb[i])
            d.parent = self.parent[i].ctypes.data_as(C.POINTER(C.c_int8))
            d.hinge_axis = self.axis[i].ctypes.data_as(C.POINTER(C.c_int8))
            d.exclude = self.exclude[i].ctypes.data_as(C.POINTER(C.c_uint64))
            d.joint_frame = self.joint_frame[i].ctypes.data_as(f)
            d.half_size = self.half[i].ctypes.data_as(f)
            d.box_center = self.com[i].ctypes.data_as(f)
            d.mass = self.mass[i].ctypes.data_as(f)
            d.cpg_w_internal = self.w_int[i].ctypes.data_as(f)
            d.cpg_w_couple = self.w_cpl[i].ctypes.data_as(f)
            d.geom = self.geom[i].ctypes.data_as(C.POINTER(C.c_int8))


def state_rows(pop: popmod.Population, q, v, s):
    """Host rows with the ABI strides (float32)."""
    n = pop.n
    Q = np.zeros((n, SIM_QW), np.float32)
    V = np.zeros((n, SIM_VW), np.float32)
    S = np.zeros((n, SIM_SW), np.float32)
    q = np.asarray(q)
    v = np.asarray(v)
    s = np.asarray(s)
    for i in range(n):
        nq, nv, ns = int(pop.nb[i]) + 6, int(pop.nb[i]) + 5, 2 * (int(pop.nb[i]) - 1)
        Q[i, :nq] = q[i, :nq]
        V[i, :nv] = v[i, :nv]
        S[i, :ns] = s[i, :ns]
    return Q, V, S


class Sim:
    """One simulation context on one CUDA device."""

    def __init__(self, **cfg):
        c = dict(DEFAULTS)
        c.update(cfg)
        self.cfg = c
        sc = SimConfig()
        for k, val in c.items():
            if k == "gravity":
                for i in range(3):
                    sc.gravity[i] = val[i]
            else:
                setattr(sc, k, val)
        h = C.c_void_p()
        rc = lib().sim_create(C.byref(sc), C.byref(h))
        if rc != 0:
            raise SimError(f"sim_create: {STATUS.get(rc, rc)}: {lib().sim_last_error(None).decode()}")
        self.h = h
        self.n = 0
        self._pop = None

    def _check(self, rc, what):
        if rc != 0:
            msg = lib().sim_last_error(self.h).decode()
            raise SimError(f"{what}: {STATUS.get(rc, rc)}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            lib().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_population(self, pop: popmod.Population):
        p32 = Population32(pop)
        self._check(lib().sim_set_population(self.h, p32.descs, pop.n), "sim_set_population")
        self._pop = pop
        self.n = pop.n

    def set_state(self, Q, V, S=None, first: int = 0):
        Q = np.ascontiguousarray(Q, np.float32)
        V = np.ascontiguousarray(V, np.float32)
        S = None if S is None else np.ascontiguousarray(S, np.float32)
        count = Q.shape[0]
        assert Q.shape[1] == SIM_QW and V.shape == (count, SIM_VW)
        assert S is None or S.shape == (count, SIM_SW)
        self._check(lib().sim_set_state(self.h, first, count, _ptr(Q), _ptr(V), _ptr(S)), "sim_set_state")

    def set_state_ptr(self, first, count, q_ptr, v_ptr, s_ptr):
        """Host pointers (e.g. pinned torch tensors) with the ABI strides."""
        self._check(lib().sim_set_state(self.h, first, count, C.c_void_p(q_ptr), C.c_void_p(v_ptr),
                                        C.c_void_p(s_ptr) if s_ptr else None), "sim_set_state")

    def step(self, n_steps: int):
        self._check(lib().sim_step_n(self.h, int(n_steps)), "sim_step_n")

    def read_state(self, first: int = 0, count: int | None = None):
        count = self.n - first if count is None else count
        Q = np.zeros((count, SIM_QW), np.float32)
        V = np.zeros((count, SIM_VW), np.float32)
        S = np.zeros((count, SIM_SW), np.float32)
        st = np.zeros(count, np.uint32)
        self._check(lib().sim_read_state(self.h, first, count, _ptr(Q), _ptr(V), _ptr(S), _ptr(st)),
                    "sim_read_state")
        return Q, V, S, st

    def read_state_ptr(self, first, count, q_ptr, v_ptr, s_ptr, st_ptr):
        self._check(lib().sim_read_state(self.h, first, count, C.c_void_p(q_ptr), C.c_void_p(v_ptr),
                                         C.c_void_p(s_ptr) if s_ptr else None,
                                         C.c_void_p(st_ptr) if st_ptr else None), "sim_read_state")

    def set_state_dev(self, first, count, q_ptr, v_ptr, s_ptr=0):
        """Device pointers (e.g. CUDA torch tensors' data_ptr()) with the ABI
        strides; queued on the context stream, no synchronisation."""
        self._check(lib().sim_set_state_dev(self.h, first, count, C.c_void_p(q_ptr), C.c_void_p(v_ptr),
                                            C.c_void_p(s_ptr) if s_ptr else None), "sim_set_state_dev")

    def read_state_dev(self, first, count, q_ptr=0, v_ptr=0, s_ptr=0, st_ptr=0):
        """Device-pointer outputs (0 = skip); queued on the context stream."""
        vp = lambda x: C.c_void_p(x) if x else None
        self._check(lib().sim_read_state_dev(self.h, first, count, vp(q_ptr), vp(v_ptr), vp(s_ptr), vp(st_ptr)),
                    "sim_read_state_dev")

    def fitness_dev(self, out_ptr, n: int | None = None):
        """Fitness of variants [0, n) into a device buffer; queued on the context stream."""
        n = self.n if n is None else n
        self._check(lib().sim_fitness_dev(self.h, C.c_void_p(out_ptr), n), "sim_fitness_dev")

    @property
    def stream(self) -> int:
        """The context's cudaStream_t as an integer (e.g. for torch.cuda.ExternalStream)."""
        s = C.c_uint64()
        self._check(lib().sim_stream(self.h, C.byref(s)), "sim_stream")
        return s.value

    def fitness(self, n: int | None = None):
        n = self.n if n is None else n
        out = np.zeros(n, np.float32)
        self._check(lib().sim_fitness(self.h, _ptr(out), n), "sim_fitness")
        return out

    def autotune(self, probe_steps: int = 50):
        self._check(lib().sim_autotune(self.h, int(probe_steps)), "sim_autotune")

    def counters(self) -> dict:
        c = Counters()
        self._check(lib().sim_counters_read(self.h, C.byref(c)), "sim_counters_read")
        return dict(contacts=c.contacts, narrow_pairs=c.narrow_pairs, broad_pairs=c.broad_pairs,
                    variant_steps=c.variant_steps, sm_cycles=c.sm_cycles)

    def debug_contacts(self, i: int, max_contacts: int = 64):
        rows = np.zeros((max_contacts, 8), np.float32)
        bb = np.zeros(max_contacts, np.int32)
        n = C.c_int32(0)
        self._check(lib().sim_debug_contacts(self.h, i, max_contacts, _ptr(rows), _ptr(bb), C.byref(n)),
                    "sim_debug_contacts")
        m = min(n.value, max_contacts)
        return dict(n=n.value, p=rows[:m, 0:3], nrm=rows[:m, 3:6], depth=rows[:m, 6],
                    a=rows[:m, 7].astype(np.int32), b=bb[:m])

    def launch_shape(self) -> dict:
        """Launch shape in use (warps per block, phase lock, steps per launch,
        resident warps per SM)."""
        w, lk, spl, occ = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self._check(lib().sim_launch_shape(self.h, C.byref(w), C.byref(lk), C.byref(spl), C.byref(occ)),
                    "sim_launch_shape")
        return dict(warps_per_block=w.value, phase_lock=lk.value, steps_per_launch=spl.value,
                    warps_per_sm=occ.value)

    def robot_cost(self):
        """SM cycles per step of every robot in the last launch (caller order)."""
        out = np.zeros(self.n, np.float32)
        self._check(lib().sim_robot_cost(self.h, _ptr(out), self.n), "sim_robot_cost")
        return out

    def debug_solver(self, i: int):
        vfree = np.zeros(SIM_VW, np.float32)
        lam = np.zeros(3 * SIM_MAX_CONTACT_CAP, np.float32)
        n = C.c_int32(0)
        cyc = np.zeros(11, np.float32)
        self._check(lib().sim_debug_solver(self.h, i, _ptr(vfree), _ptr(lam), C.byref(n), _ptr(cyc)),
                    "sim_debug_solver")
        return dict(vfree=vfree, lam=lam[:3 * n.value].reshape(-1, 3), n=n.value,
                    cycles_per_step=float(cyc[0]), phase_cycles=cyc[1:10].copy())


def fp32_peak(device: int = 0, launches: int = 25) -> dict:
    """FP32 FMA throughput of the device measured by the library's FFMA-loop
    kernel: FLOP count, device milliseconds, TFLOP/s and SM count."""
    fl, ms, sms = C.c_double(), C.c_float(), C.c_int32()
    rc = lib().sim_fp32_peak(device, launches, C.byref(fl), C.byref(ms), C.byref(sms))
    if rc != 0:
        raise SimError(f"sim_fp32_peak: {STATUS.get(rc, rc)}: {lib().sim_last_error(None).decode()}")
    return dict(flops=fl.value, ms=ms.value, tflops=fl.value / (ms.value * 1e-3) / 1e12, sms=sms.value)


def debug_sincos(x):
    """The step kernel's FP64 sine / cosine routine evaluated on the host."""
    x = np.ascontiguousarray(x, np.float64)
    s = np.zeros_like(x)
    c = np.zeros_like(x)
    rc = lib().sim_debug_sincos(_ptr(x), x.size, _ptr(s), _ptr(c))
    if rc != 0:
        raise SimError(f"sim_debug_sincos: {rc}")
    return s, c
