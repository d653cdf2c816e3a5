"""The C-ABI library loads and exports every entry point of include/*.h.

No compute calls here (no GPU needed): only symbol presence and the argument
checks that fail before any device is touched.
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2502_11129_b300 import build as B
from paper_2502_11129_b300 import sim as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z][a-z0-9_]*)\s*\(", text, re.M):
            names.setdefault(os.path.basename(h), []).append(m.group(1))
    return names


def test_libraries_build_and_export_every_declared_symbol():
    B.build()
    decl = header_functions()
    assert "b3sim.h" in decl and len(decl["b3sim.h"]) >= 11
    from paper_2502_11129_b300 import cpu as CP
    from paper_2502_11129_b300 import surrogate as SG
    libs = {"b3sim.h": S.LIB_PATH, "b3sur.h": SG.LIB_PATH, "b3cpu.h": CP.LIB_PATH}
    for header, names in decl.items():
        assert header in libs, f"no library for {header}"
        L = C.CDLL(libs[header])
        missing = [n for n in names if not hasattr(L, n)]
        assert not missing, (header, missing)


def test_binding_lists_every_declared_entry_point():
    from paper_2502_11129_b300 import cpu as CP
    from paper_2502_11129_b300 import surrogate as SG
    decl = header_functions()
    assert sorted(decl["b3sim.h"]) == sorted(S.EXPORTS)
    assert sorted(decl["b3sur.h"]) == sorted(SG.EXPORTS)
    assert sorted(decl["b3cpu.h"]) == sorted(CP.EXPORTS)


def test_sim_create_argument_errors_without_device():
    L = S.lib()
    h = C.c_void_p()
    assert L.sim_create(None, C.byref(h)) == -1
    assert b"NULL" in L.sim_last_error(None)
    cfg = S.SimConfig()
    for k, v in S.DEFAULTS.items():
        if k == "gravity":
            for i in range(3):
                cfg.gravity[i] = v[i]
        else:
            setattr(cfg, k, v)
    cfg.contact_cap = 1000
    assert L.sim_create(C.byref(cfg), C.byref(h)) == -1
    assert h.value is None
    cfg.contact_cap = 64
    cfg.pgs_iters = 0
    assert L.sim_create(C.byref(cfg), C.byref(h)) == -1
    assert L.sim_destroy(None) == 0


def test_null_context_is_rejected():
    L = S.lib()
    assert L.sim_step_n(None, 1) == -1
    assert L.sim_set_population(None, None, 0) == -1
    assert L.sim_read_state(None, 0, 0, None, None, None, None) == -1


def test_step_kernel_fp64_sincos_against_libm():
    """The hinge-angle sine / cosine routine of the step kernel (host build of
    the same source) against the platform libm: absolute error within 4e-16
    on |x| <= 10 and within 1e-15 on |x| <= 1e5."""
    rng = np.random.default_rng(0)
    for lim, tol in ((10.0, 4e-16), (1e5, 1e-15)):
        x = np.concatenate([rng.uniform(-lim, lim, 200000), np.linspace(-lim, lim, 10001),
                            np.pi / 2 * np.arange(-6, 7), [0.0, -0.0, 1e-300]])
        s, c = S.debug_sincos(x)
        assert np.abs(s - np.sin(x)).max() <= tol
        assert np.abs(c - np.cos(x)).max() <= tol
    assert S.lib().sim_debug_sincos(None, 1, None, None) == -1  # SIM_EINVAL


def test_binding_constants_match_the_header():
    """Row strides and body bounds of the binding are those of include/b3sim.h."""
    text = open(os.path.join(ROOT, "include", "b3sim.h")).read()
    val = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(SIM_[A-Z_]+)\s+(\d+)", text)}
    assert val["SIM_MAX_BODIES"] == S.SIM_MAX_BODIES == 64
    assert val["SIM_WARP_MAX_BODIES"] == S.SIM_WARP_MAX_BODIES
    assert (val["SIM_QW"], val["SIM_VW"], val["SIM_SW"]) == (S.SIM_QW, S.SIM_VW, S.SIM_SW)
    # rows hold the largest robot: nq = nb + 6, nv = nb + 5, 2 (nb - 1) CPG states
    assert S.SIM_QW >= S.SIM_MAX_BODIES + 6 and S.SIM_VW >= S.SIM_MAX_BODIES + 5
    assert S.SIM_SW >= 2 * (S.SIM_MAX_BODIES - 1)
    assert val["SIM_MAX_CONTACT_CAP"] == S.SIM_MAX_CONTACT_CAP
