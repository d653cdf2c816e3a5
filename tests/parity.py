"""One-step parity of an FP32 engine against the FP64 oracle (test helper).

From identical FP32-rounded states, per robot:
  e_norm  max over x in (q, v, s) of |x_eng - x_ref| / max(|x_ref|, 1), the
          stated per-step bar (Euclidean norms over the robot's entries);
  e_elem  max over every entry i of q, v, s of
          |x_eng,i - x_ref,i| / max(|x_ref,i|, 1), the worst single entry.
x_ref is the oracle's step.  Where the step takes a discrete decision within
BAND of its threshold (contact activation, separating-axis or incident-face
choice, clipping side, cap cut, frozen rows), FP32 and FP64 arithmetic may
legitimately go either way: every valid outcome of the step (the oracle with
those decisions taken either way, oracle.step_outcomes) is a reference, and
the engine is compared with the closest one.  No robot is left out, and no
reference value comes from the engine.

The FP32 yardstick (oracle32: the same oracle source evaluated in FP32) gives
the spread that FP32 arithmetic alone brings to one step of the method on the
same states; where the FP64 result is ill-conditioned (settled, servo-loaded
robots, long chains) no FP32 implementation of the method meets 1e-5 on every
robot, and the engine is held to that yardstick instead.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

from oracle import oracle as O
from oracle import oracle32 as O32

BAND = 1e-5
TOL_STEP = 1e-5          # the stated per-step bar
CAP_NORM = 5e-5          # ceiling per robot where FP32 itself cannot meet TOL_STEP
CAP_ELEM = 1e-4          # ceiling of the worst single entry per robot
SAME_SCALE = 2.0         # two FP32 evaluations of one step: quantiles within this factor
TAIL_SCALE = 4.0         # ... and their worst robots (the largest of a few dozen
                         # heavy-tailed samples: two correct FP32 engines differ by ~2x there)
ORACLE_KEYS = ("dt", "gravity", "pgs_iters", "mu", "contact_cap", "ground", "box_box", "actuate", "armature",
               "max_correct_vel", "min_cfm")


def ncores():
    return max(1, len(os.sched_getaffinity(0)))


def oracle_params(**cfg):
    return O.default_params(**{k: v for k, v in cfg.items() if k in ORACLE_KEYS})


@dataclass
class StepErrors:
    e_norm: np.ndarray      # per robot
    e_elem: np.ndarray      # per robot
    parts: np.ndarray       # per robot: norms of q, v, s
    n_near: np.ndarray      # near-threshold decisions of the oracle's step
    status_ref: np.ndarray  # status bits of the closest outcome

    def summary(self, name: str) -> str:
        def q(x):
            return f"median {np.median(x):.2e} p90 {np.quantile(x, 0.9):.2e} max {x.max():.2e}"
        return (f"{name}: n={len(self.e_norm)} near-threshold={int((self.n_near > 0).sum())} "
                f"norm[{q(self.e_norm)}] elem[{q(self.e_elem)}] worst q,v,s={self.parts.max(axis=0)} "
                f"over-1e-5={np.nonzero(self.e_norm > TOL_STEP)[0][:12].tolist()}")


def _errors(nq, nv, ns, eq, ev, es, ref):
    oq, ov, os_ = ref[0][:nq], ref[1][:nv], ref[2][:ns]
    parts = np.array([np.linalg.norm(eq[:nq] - oq) / max(np.linalg.norm(oq), 1.0),
                      np.linalg.norm(ev[:nv] - ov) / max(np.linalg.norm(ov), 1.0),
                      np.linalg.norm(es[:ns] - os_) / max(np.linalg.norm(os_), 1.0) if ns else 0.0])
    el = 0.0
    for a, b in ((eq[:nq], oq), (ev[:nv], ov), (es[:ns], os_)):
        if len(b):
            el = max(el, float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))))
    return parts, el


def one_step_errors(pop32, Q, V, Sx, eq, ev, es, prm=None) -> StepErrors:
    """Errors of an engine's one-step result (eq, ev, es: rows with the ABI
    strides) against the closest valid outcome of the oracle's step from the
    same FP32 states (Q, V, Sx)."""
    prm = prm or O.default_params()
    n = pop32.n
    e_norm = np.zeros(n)
    e_elem = np.zeros(n)
    parts = np.zeros((n, 3))
    n_near = np.zeros(n, np.int64)
    st_ref = np.zeros(n, np.uint32)
    for i in range(n):
        m = O.model_from_population(pop32, i)
        nq, nv, ns = O.nq(m), O.nv(m), 2 * (m.nb - 1)
        s64 = np.zeros(2 * O.MAXB)
        s64[:ns] = Sx[i, :ns]
        outs, k, _ = O.step_outcomes(m, Q[i, :nq].astype(np.float64), V[i, :nv].astype(np.float64), s64,
                                     band=BAND, prm=prm)
        best = None
        for ref in outs:
            p, el = _errors(nq, nv, ns, np.asarray(eq[i], np.float64), np.asarray(ev[i], np.float64),
                            np.asarray(es[i], np.float64), ref)
            key = (p.max(), el)
            if best is None or key < best[0]:
                best = (key, p, el, ref[3])
        (e_norm[i], e_elem[i]), parts[i], st_ref[i] = best[0], best[1], best[3]
        n_near[i] = k
    return StepErrors(e_norm, e_elem, parts, n_near, st_ref)


def fp32_yardstick(pop32, Q, V, Sx, prm=None) -> StepErrors:
    """The same errors for the oracle's own FP32 build on the same states."""
    prm = prm or O.default_params()
    fq, fv, fs, _, _ = O32.run_population(pop32, Q, V, Sx, 1, prm=prm, threads=ncores())
    return one_step_errors(pop32, Q, V, Sx, fq, fv, fs, prm)


def parity_failures(r: StepErrors, y: StepErrors) -> list[str]:
    """The bars, fixed before any engine result is seen:
      * where FP32 arithmetic meets the stated per-step bar on every robot of
        these states (the yardstick y does), the engine must too: e_norm <=
        1e-5 for every robot;
      * elsewhere (ill-conditioned states) the engine's e_norm distribution
        must be that of FP32 arithmetic: median and 90th percentile within
        SAME_SCALE of the yardstick's (two FP32 evaluations of one step differ
        in their rounding, not in their scale), and every robot under
        CAP_NORM or TAIL_SCALE times the yardstick's worst robot, whichever
        is larger (long chains);
      * the worst single entry likewise: e_elem median and 90th percentile
        within SAME_SCALE of the yardstick's, every robot under CAP_ELEM or
        TAIL_SCALE times the yardstick's worst robot.
    Returns the failed criteria (empty: pass)."""
    bad = []
    if (y.e_norm <= TOL_STEP).all():
        if (r.e_norm > TOL_STEP).any():
            bad.append(f"norm above {TOL_STEP} (FP32 meets it here): {np.nonzero(r.e_norm > TOL_STEP)[0][:10].tolist()}")
    else:
        for qq in (0.5, 0.9):
            if np.quantile(r.e_norm, qq) > SAME_SCALE * np.quantile(y.e_norm, qq):
                bad.append(f"norm q{qq}: {np.quantile(r.e_norm, qq):.3g} > {SAME_SCALE} x fp32 "
                           f"{np.quantile(y.e_norm, qq):.3g}")
        cap = max(CAP_NORM, TAIL_SCALE * y.e_norm.max())
        if (r.e_norm > cap).any():
            bad.append(f"norm above {cap:.3g}: {np.nonzero(r.e_norm > cap)[0][:10].tolist()}")
    for qq in (0.5, 0.9):
        if np.quantile(r.e_elem, qq) > SAME_SCALE * np.quantile(y.e_elem, qq):
            bad.append(f"elem q{qq}: {np.quantile(r.e_elem, qq):.3g} > {SAME_SCALE} x fp32 "
                       f"{np.quantile(y.e_elem, qq):.3g}")
    cap = max(CAP_ELEM, TAIL_SCALE * y.e_elem.max())
    if (r.e_elem > cap).any():
        bad.append(f"elem above {cap:.3g}: {np.nonzero(r.e_elem > cap)[0][:10].tolist()}")
    return bad
