"""Python binding of include/b3sur.h (argument marshalling only).

The surrogate's arithmetic (encoding, the BF16 tensor-core MLP, its training
and the top-k selection) runs in ``libb3sur.so``; this module converts numpy
arrays to pointers.  No CPU fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libb3sur.so")
IN_DIM, HIDDEN = 128, 256
NPARAMS = HIDDEN * IN_DIM + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1
MAX_BATCH, MAX_TOPK = 65536, 8192
EXPORTS = ["sur_create", "sur_destroy", "sur_encode", "sur_train", "sur_predict", "sur_topk",
           "sur_gradients", "sur_train_step", "sur_get_params", "sur_set_params", "sur_last_error"]
STATUS = {0: "SUR_OK", -1: "SUR_EINVAL", -2: "SUR_ECUDA", -3: "SUR_ENOMEM"}


class SurConfig(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("device", C.c_int32), ("stream", C.c_uint64)]


class SurrogateError(RuntimeError):
    pass


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SurrogateError(f"{LIB_PATH} is missing; build it with python -m paper_2502_11129_b300.build")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.sur_create.argtypes = [C.POINTER(SurConfig), C.POINTER(vp)]
        L.sur_destroy.argtypes = [vp]
        L.sur_encode.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int32, vp]
        L.sur_train.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, vp]
        L.sur_predict.argtypes = [vp, vp, C.c_int32, vp]
        L.sur_topk.argtypes = [vp, vp, C.c_int32, C.c_int32, vp]
        L.sur_gradients.argtypes = [vp, vp, vp, C.c_int32, vp, vp]
        L.sur_train_step.argtypes = [vp, vp, vp, C.c_int32, vp]
        L.sur_get_params.argtypes = [vp, vp]
        L.sur_set_params.argtypes = [vp, vp]
        L.sur_last_error.argtypes = [vp]
        L.sur_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data)


def pack_params(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack_params(flat) -> dict:
    flat = np.asarray(flat)
    shapes = [("W1", (HIDDEN, IN_DIM)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
              ("W3", (1, HIDDEN)), ("b3", (1,))]
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = flat[o:o + n].reshape(sh)
        o += n
    return out


class Surrogate:
    def __init__(self, seed=0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, device=0, stream=0):
        cfg = SurConfig(seed, lr, beta1, beta2, eps, device, stream)
        h = C.c_void_p()
        rc = lib().sur_create(C.byref(cfg), C.byref(h))
        if rc != 0:
            raise SurrogateError(f"sur_create: {STATUS.get(rc, rc)}: {lib().sur_last_error(None).decode()}")
        self.h = h

    def _check(self, rc, what):
        if rc != 0:
            raise SurrogateError(f"{what}: {STATUS.get(rc, rc)}: {lib().sur_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib().sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def encode(self, pop) -> np.ndarray:
        n = pop.n
        X = np.zeros((n, IN_DIM), np.float32)
        s = pop.slots  # 32 (or 64 for long chains, which the library rejects: > 21 bodies)
        take = slice(0, 32)
        parent = np.ascontiguousarray(pop.parent[:, take], np.int8)
        axis = np.ascontiguousarray(pop.axis[:, take], np.int8)
        R_fix = np.ascontiguousarray(pop.R_fix.reshape(n, s, 9)[:, take], np.float32)
        p_fix = np.ascontiguousarray(pop.p_fix[:, take], np.float32)
        com = np.ascontiguousarray(pop.com[:, take], np.float32)
        wi = np.ascontiguousarray(pop.w_int[:, take], np.float32)
        wc = np.ascontiguousarray(pop.w_cpl[:, take], np.float32)
        nb = np.ascontiguousarray(pop.nb, np.int32)
        self._check(lib().sur_encode(self.h, _p(parent), _p(axis), _p(R_fix), _p(p_fix), _p(com), _p(wi), _p(wc),
                                     _p(nb), n, _p(X)), "sur_encode")
        return X

    def train(self, X, y, epochs=10, batch=1024) -> float:
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = C.c_float(0.0)
        self._check(lib().sur_train(self.h, _p(X), _p(y), len(y), epochs, batch, C.byref(loss)), "sur_train")
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros(X.shape[0], np.float32)
        self._check(lib().sur_predict(self.h, _p(X), X.shape[0], _p(out)), "sur_predict")
        return out

    def topk(self, scores, k) -> np.ndarray:
        s = np.ascontiguousarray(scores, np.float32)
        idx = np.zeros(k, np.int32)
        self._check(lib().sur_topk(self.h, _p(s), len(s), k, _p(idx)), "sur_topk")
        return idx

    def gradients(self, X, y):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        g = np.zeros(NPARAMS, np.float32)
        loss = C.c_float(0.0)
        self._check(lib().sur_gradients(self.h, _p(X), _p(y), len(y), _p(g), C.byref(loss)), "sur_gradients")
        return g, loss.value

    def train_step(self, X, y) -> float:
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = C.c_float(0.0)
        self._check(lib().sur_train_step(self.h, _p(X), _p(y), len(y), C.byref(loss)), "sur_train_step")
        return loss.value

    def get_params(self) -> np.ndarray:
        p = np.zeros(NPARAMS, np.float32)
        self._check(lib().sur_get_params(self.h, _p(p)), "sur_get_params")
        return p

    def set_params(self, flat):
        p = np.ascontiguousarray(flat, np.float32)
        assert p.size == NPARAMS
        self._check(lib().sur_set_params(self.h, _p(p)), "sur_set_params")


def timing(n_train=50000, n_screen=65536, k=4096, epochs=3, batch=1024, seed=0) -> dict:
    """Wall times of the screening workload's surrogate calls (cfg4 sizes) on
    synthetic genotypes; each call includes its host<->device copies."""
    import time
    from . import population as P
    rng = np.random.default_rng(seed)
    s = Surrogate(seed=seed)
    out = {}
    pop = P.grammar(2048, seed=seed)
    t = time.perf_counter()
    X = s.encode(pop)
    out["encode_2048_s"] = time.perf_counter() - t
    Xt = rng.normal(0, 0.5, (n_train, IN_DIM)).astype(np.float32)
    yt = rng.normal(0, 1, n_train).astype(np.float32)
    # warm-up at the timed size: the first call per (rows, batch) captures the
    # training epoch as a CUDA graph; the timed calls replay it
    s.train(Xt, yt, epochs=1, batch=batch)
    t = time.perf_counter()
    s.train(Xt, yt, epochs=1, batch=batch)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    s.train(Xt, yt, epochs=epochs, batch=batch)
    dt = time.perf_counter() - t
    out["train_s_per_epoch"] = (dt - t1) / (epochs - 1) if epochs > 1 else dt
    # forward + backward GEMM flops of one sample: 3 x 2 x (128*256 + 256*256 + 256)
    fl = 6.0 * (IN_DIM * HIDDEN + HIDDEN * HIDDEN + HIDDEN)
    out.update(train_epochs=epochs, train_s=dt, train_samples_per_s=n_train * epochs / dt,
               train_tflops_incl_host=fl * n_train * epochs / dt / 1e12)
    Xs = rng.normal(0, 0.5, (n_screen, IN_DIM)).astype(np.float32)
    s.predict(Xs[:1024])
    t = time.perf_counter()
    y = s.predict(Xs)
    dt = time.perf_counter() - t
    out.update(predict_n=n_screen, predict_s=dt, predict_per_s=n_screen / dt,
               predict_tflops_incl_host=2.0 * (IN_DIM * HIDDEN + HIDDEN * HIDDEN + HIDDEN) * n_screen / dt / 1e12)
    t = time.perf_counter()
    s.topk(y, k)
    out["topk_s"] = time.perf_counter() - t
    s.close()
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(timing()))
