"""Allocation-free stepping against the context-based entry point.

sim_step_n_noalloc exists for callers that cannot allocate device memory when
they step: hosts whose device memory is owned by another allocator or fixed up
front (a cudaMalloc would bypass their accounting or fail against their
budget), and real-time loops that must not block in the driver (cudaMalloc and
cudaFree may synchronise the device).  They keep the population in device
buffers they already own; the library's per-variant scratch comes from a fixed
array inside the library.

This test packs a population in the documented device layout (include/b3sim.h),
steps it twice in a row through sim_step_n_noalloc, and compares both results
with sim_step_n on the same population.  It lives in its own file, collected
last, so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import sim as S

pytestmark = pytest.mark.gpu

NF, NI = 26, 5
TOL = 1e-6


def pack(pop):
    """Device layout of sim_device_population (see include/b3sim.h)."""
    p32 = S.Population32(pop)
    n = pop.n
    mf = np.zeros((n, NF, 32), np.float32)
    mi = np.zeros((n, NI, 32), np.int32)
    meta = np.zeros((n, 4), np.int32)
    pairs = []
    for i in range(n):
        nb = int(pop.nb[i])
        mf[i, 0, :] = 1.0
        mf[i, 4, :] = 1.0
        mf[i, 8, :] = 1.0
        mi[i, 0, :] = -1
        depth = np.zeros(32, np.int32)
        path = np.zeros(32, np.uint32)
        child = np.zeros(32, np.uint32)
        parent = [int(x) for x in p32.parent[i]]
        for b in range(nb):
            p = -1 if b == 0 else parent[b]
            depth[b] = 0 if p < 0 else depth[p] + 1
            path[b] = (0 if p < 0 else path[p]) | np.uint32(1 << b)
            if p >= 0:
                child[p] |= np.uint32(1 << b)
        for b in range(nb):
            mf[i, 0:9, b] = p32.joint_frame[i, b, 0:9]
            mf[i, 9:12, b] = p32.joint_frame[i, b, 9:12]
            mf[i, 12:15, b] = p32.half[i, b]
            mf[i, 15:18, b] = p32.com[i, b]
            m = float(p32.mass[i, b])
            hx, hy, hz = (float(x) for x in p32.half[i, b])
            sphere = int(p32.geom[i, b]) == P.GEOM_SPHERE
            mf[i, 18, b] = p32.mass[i, b]
            if sphere:
                mf[i, 19:22, b] = np.float32(0.4 * m * hx * hx)
            else:
                mf[i, 19, b] = np.float32(m * (hy * hy + hz * hz) / 3.0)
                mf[i, 20, b] = np.float32(m * (hx * hx + hz * hz) / 3.0)
                mf[i, 21, b] = np.float32(m * (hx * hx + hy * hy) / 3.0)
            mf[i, 22, b] = p32.w_int[i, b]
            mf[i, 23, b] = p32.w_cpl[i, b]
            mf[i, 24, b] = np.float32(hx) if sphere else np.float32(np.sqrt(hx * hx + hy * hy + hz * hz))
            mf[i, 25, b] = 1.0 if sphere else 0.0
            mi[i, 0, b] = -1 if b == 0 else parent[b]
            mi[i, 1, b] = int(p32.axis[i, b])
            mi[i, 2, b] = np.int32(path[b].view(np.int32))
            mi[i, 3, b] = np.int32(child[b].view(np.int32))
            mi[i, 4, b] = depth[b]
        off = len(pairs)
        ex = [int(x) for x in p32.exclude[i]]
        for a in range(nb):
            for b in range(a + 1, nb):
                if parent[b] == a or (ex[a] >> b) & 1 or (ex[b] >> a) & 1:
                    continue
                pairs.append((a << 8) | b)
        meta[i] = (nb, int(depth[:nb].max()), len(pairs) - off, off)
    if not pairs:
        pairs = [0]
    return mf, mi, meta, np.array(pairs, np.uint16)


def config(**kw):
    c = dict(S.DEFAULTS)
    c.update(kw)
    sc = S.SimConfig()
    for k, v in c.items():
        if k == "gravity":
            for j in range(3):
                sc.gravity[j] = v[j]
        else:
            setattr(sc, k, v)
    return sc


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


def _device_pop(pop, Q, V, Sx):
    import torch
    dev = torch.device("cuda", 0)
    mf, mi, meta, pairs = pack(pop)
    # the device rows of this layout are 32, 32 and 64 floats wide (the host rows are wider)
    t = {k: torch.from_numpy(np.ascontiguousarray(a)).to(dev) for k, a in
         dict(mf=mf, mi=mi, meta=meta, pairs=pairs.view(np.int16), q=Q[:, :32], v=V[:, :32],
              s=Sx[:, :64]).items()}
    t["st"] = torch.zeros(pop.n, dtype=torch.int32, device=dev)
    dp = S.DevicePopulation(pop.n, t["mf"].data_ptr(), t["mi"].data_ptr(), t["meta"].data_ptr(),
                            t["pairs"].data_ptr(), t["q"].data_ptr(), t["v"].data_ptr(), t["s"].data_ptr(),
                            t["st"].data_ptr())
    return t, dp


def test_noalloc_matches_context_entry_on_two_calls():
    import torch

    pop = P.grammar(48, seed=17, ball_p=0.25).as_float32()  # geometry field too
    q, v, s = P.random_state(pop, seed=3, angle=0.4)
    q[:, 2] = pop.q0[:, 2] - 0.004
    Q, V, Sx = S.state_rows(pop, q, v, s)

    ref = S.Sim()
    ref.set_population(pop)
    ref.set_state(Q, V, Sx)

    dev = torch.device("cuda", 0)
    t, dp = _device_pop(pop, Q, V, Sx)
    cfg = config(stream=0)
    L = S.lib()
    for call in range(2):
        rc = L.sim_step_n_noalloc(C.byref(cfg), C.byref(dp), 60)
        assert rc == 0, L.sim_last_error(None)
        torch.cuda.synchronize(dev)
        ref.step(60)
        rq, rv, rs, rst = ref.read_state()
        rq, rv, rs = rq[:, :32], rv[:, :32], rs[:, :64]
        gq, gv, gs = t["q"].cpu().numpy(), t["v"].cpu().numpy(), t["s"].cpu().numpy()
        gst = t["st"].cpu().numpy().view(np.uint32)
        assert np.array_equal(gst, rst), call
        assert rel_err(gq, rq) <= TOL, (call, rel_err(gq, rq))
        assert rel_err(gv, rv) <= TOL, (call, rel_err(gv, rv))
        assert rel_err(gs, rs) <= TOL, (call, rel_err(gs, rs))
        assert np.abs(gq[:, :3] - Q[:, :3]).max() > 0  # the robots did move
    ref.close()


def test_noalloc_single_free_bodies_take_the_general_kernel():
    """Free cubes: sim_step_n steps them one thread per body, this entry point
    with the general warp kernel; the two agree to FP32 rounding (the bar of
    the CPU engine's one-body / general-step comparison), on two calls."""
    import torch

    pop = P.boxes(24, seed=13, vel_sigma=2.0).as_float32()
    q = pop.q0.copy()
    q[:, 2] = np.random.default_rng(14).uniform(0.02, 0.3, pop.n)
    Q, V, Sx = S.state_rows(pop, q, pop.v0, np.zeros((pop.n, 64)))
    ref = S.Sim()
    ref.set_population(pop)
    ref.set_state(Q, V, Sx)
    dev = torch.device("cuda", 0)
    t, dp = _device_pop(pop, Q, V, Sx)
    cfg = config(stream=0)
    L = S.lib()
    for call in range(2):
        assert L.sim_step_n_noalloc(C.byref(cfg), C.byref(dp), 100) == 0, L.sim_last_error(None)
        torch.cuda.synchronize(dev)
        ref.step(100)
        rq, rv, _, rst = ref.read_state()
        gq, gv = t["q"].cpu().numpy(), t["v"].cpu().numpy()
        gst = t["st"].cpu().numpy().view(np.uint32)
        assert np.array_equal(gst, rst) and (gst & 5).sum() == 0, call
        assert np.abs(gq[:, :7] - rq[:, :7]).max() < 5e-5, call
        assert np.abs(gv[:, :6] - rv[:, :6]).max() < 1e-4 * max(1.0, np.abs(rv[:, :6]).max()), call
    ref.close()


def test_noalloc_rejects_more_variants_than_its_scratch():
    L = S.lib()
    dp = S.DevicePopulation(S_MAX + 1, 16, 16, 16, 16, 16, 16, 16, 16)
    cfg = config()
    assert L.sim_step_n_noalloc(C.byref(cfg), C.byref(dp), 1) == -1
    assert b"64" in L.sim_last_error(None)


def test_noalloc_rejects_a_misaligned_meta_buffer():
    """The meta rows are read as 16-byte vectors: a buffer at a 4-byte offset
    is refused on the host, before anything is launched."""
    L = S.lib()
    dp = S.DevicePopulation(4, 256, 256, 256 + 4, 256, 256, 256, 256, 256)
    cfg = config()
    assert L.sim_step_n_noalloc(C.byref(cfg), C.byref(dp), 1) == -1
    assert b"aligned" in L.sim_last_error(None)


S_MAX = 64
