"""ctypes binding of the learned form of the C++ oracle
(``oracle/qtt_oracle.cpp``): the rank features, the MLP forward and
backward passes, Adam, the randomised range finder with its exact
acceptance check, and the round that uses it.

TEST INFRASTRUCTURE ONLY: only ``tests/`` use it.  It offers the names and
formats of ``oracle/learned.py`` so that the same pins run on both oracles,
but shares no arithmetic with it: every function below calls the C++ code.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from oracle import cxx as X

N_FEAT = 40
WIDTH = 128
OVERSAMPLE = 16
TAU = 0.05
SHAPES = [(WIDTH, N_FEAT), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (1, WIDTH), (1,)]

_sigs_done = False


def _lib():
    global _sigs_done
    lib = X._load()
    if not _sigs_done:
        i, d, dp, ip, vp = C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p
        for name, res, args in (
                ("oc_mlp_param_count", i, []),
                ("oc_rank_features", None, [dp, i, i, d, i, i, i, dp]),
                ("oc_mlp_forward", None, [dp, dp, i, dp]),
                ("oc_mlp_grad", d, [dp, dp, dp, i, dp]),
                ("oc_adam_step", None, [dp, dp, dp, dp, i, i, d, d, d, d]),
                ("oc_range_finder_svd", i, [i, i, dp, i, dp, d, i, d, ip, dp, dp, dp, ip, dp]),
                ("oc_round_learned", vp, [vp, d, i, ip, i, i, dp, i, d, ip, ip])):
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _sigs_done = True
    return lib


N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)  # the flat layout; the C++ side reports the same count


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def unpack(flat: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts: list[np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def rank_features(S, r: int, eps: float, chi: int, k: int, d: int) -> np.ndarray:
    S = _f64(S)
    f = np.zeros(N_FEAT)
    _lib().oc_rank_features(X._dp(S), S.size, int(r), float(eps), int(chi), int(k), int(d), X._dp(f))
    return f


def mlp_forward(params: np.ndarray, Xf: np.ndarray):
    p, x = _f64(params), _f64(Xf)
    y = np.zeros(x.shape[0])
    _lib().oc_mlp_forward(X._dp(p), X._dp(x), x.shape[0], X._dp(y))
    return y, {}


def mse_loss(y, t) -> float:
    return float(np.mean((np.asarray(y) - np.asarray(t)) ** 2))


def mlp_grad(params: np.ndarray, Xf: np.ndarray, t) -> tuple[float, np.ndarray]:
    p, x, tt = _f64(params), _f64(Xf), _f64(t)
    g = np.zeros(p.size)
    loss = _lib().oc_mlp_grad(X._dp(p), X._dp(x), X._dp(tt), x.shape[0], X._dp(g))
    return float(loss), g


def adam_step(params, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    p, gg, mm, vv = _f64(params).copy(), _f64(g), _f64(m).copy(), _f64(v).copy()
    _lib().oc_adam_step(X._dp(p), X._dp(gg), X._dp(mm), X._dp(vv), p.size, int(t), float(lr), float(beta1),
                        float(beta2), float(eps))
    return p, mm, vv


def propose_rank(y: float, chi: int) -> int:
    """r_hat = ceil(chi * y), clamped to [1, chi] (host rule, as in the library's binding)."""
    return int(min(max(int(np.ceil(chi * y)), 1), chi))


def range_finder_svd(Xm: np.ndarray, Omega: np.ndarray, eps: float, chi: int, tau: float = TAU):
    x, om = _f64(Xm), _f64(Omega)
    l, m = x.shape
    ks = om.shape[1]
    q = min(m, ks)
    Vt, US, Sb = np.zeros(q * m), np.zeros(l * q), np.zeros(q)
    r, nsb, rho = C.c_int(0), C.c_int(0), C.c_double(0.0)
    ok = _lib().oc_range_finder_svd(l, m, X._dp(x), ks, X._dp(om), float(eps), int(chi), float(tau), C.byref(r),
                                    X._dp(Vt), X._dp(US), X._dp(Sb), C.byref(nsb), C.byref(rho))
    r = r.value
    return bool(ok), r, Vt[:r * m].reshape(r, m), US[:l * r].reshape(l, r), Sb[:nsb.value], rho.value


def tt_round_learned(A: list[np.ndarray], eps: float, chi: int, proposals, G: np.ndarray, p: int = OVERSAMPLE,
                     tau: float = TAU, stats=None, log: list | None = None) -> list[np.ndarray]:
    lib = _lib()
    h = X._Mps.of(A)
    d = len(A)
    props = None if proposals is None else np.ascontiguousarray(proposals, dtype=np.int32)
    g = _f64(G)
    lg = np.zeros(3 * d, dtype=np.int32)
    nlog = C.c_int(0)
    out = X._Mps(lib.oc_round_learned(h.h, float(eps), int(chi), None if props is None else X._ip(props),
                                      g.shape[0], g.shape[1], X._dp(g), int(p), float(tau), X._ip(lg),
                                      C.byref(nlog)))
    if log is not None:
        for j in range(0, nlog.value, 3):
            log.append((int(lg[j]), int(lg[j + 1]), bool(lg[j + 2])))
    return out.cores()



def param_count() -> int:
    """Parameter count of the C++ oracle's network."""
    return int(_lib().oc_mlp_param_count())
