"""ctypes binding of the C++ oracle (``oracle/qtt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only ``tests/`` use it.  It marshals numpy arrays to the
C++ oracle and back, in the formats of the numpy oracle (MPS cores
``[r_{k-1}][2][r_k]``, MPO cores ``[w_{k-1}][t][s][w_k]``, dense fields
``u[x, z]``), so that tests can pin it and compare the two oracles.  The C++
oracle has its own Householder QR and one-sided Jacobi SVD and uses no BLAS or
LAPACK.

The library is built with g++ (no GPU compiler) into ``oracle/`` on first use,
or by :func:`build`, and rebuilt when the source is newer.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtt_oracle.cpp")
_LIB = os.path.join(_HERE, "libqtt_oracle_cxx.so")

_ORDER = {"sequential": 0, "interleaved": 1}
_BC = {"periodic": 0, "zero": 1}
_AXIS = {"x": 0, "z": 1}

_lib = None


def build(force: bool = False) -> str:
    """Compile the C++ oracle with g++ (portable x86-64 code, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    sig = {
        "oc_mps_from_cores": (vp, [i, ip, dp]),
        "oc_mps_sites": (i, [vp]),
        "oc_mps_ranks": (None, [vp, ip]),
        "oc_mps_data": (None, [vp, dp]),
        "oc_mps_free": (None, [vp]),
        "oc_mps_from_dense": (vp, [i, i, dp, d, i]),
        "oc_mps_to_dense": (None, [vp, i, i, dp]),
        "oc_mps_sample": (None, [vp, i, i, i, ip, ip, dp]),
        "oc_product_state": (vp, [i, i, i, i]),
        "oc_round": (vp, [vp, d, i]),
        "oc_sum": (vp, [i, dp, C.POINTER(vp)]),
        "oc_shift_mpo": (vp, [i, i, i, i, i]),
        "oc_laplacian_mpo": (vp, [i, i, i]),
        "oc_laplacian_sum_of_shifts": (vp, [i, i, i]),
        "oc_diagonal_mpo": (vp, [vp]),
        "oc_mpo_sites": (i, [vp]),
        "oc_mpo_bonds": (None, [vp, ip]),
        "oc_mpo_data": (None, [vp, dp]),
        "oc_mpo_grid_operator": (None, [vp, i, i, dp]),
        "oc_mpo_free": (None, [vp]),
        "oc_zipup_lr": (vp, [vp, vp, d, i]),
        "oc_zipup_rl": (vp, [vp, vp, d, i]),
        "oc_step": (vp, [vp, vp, d, vp, vp, d, i, i, i, d, i, i]),
        "oc_fdtd_step": (None, [i, dp, dp, dp, d, i, i, i, d, dp]),
        "oc_svd": (i, [i, i, dp, dp, dp, dp]),
        "oc_qr": (None, [i, i, dp, dp, dp]),
        "oc_trunc_rank": (i, [i, dp, d, i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# handles <-> numpy cores
# ---------------------------------------------------------------------------
class _Mps:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        if self.h:
            _load().oc_mps_free(self.h)
            self.h = None

    @classmethod
    def of(cls, cores: list[np.ndarray]) -> "_Mps":
        lib = _load()
        d = len(cores)
        ranks = np.array([cores[0].shape[0]] + [c.shape[2] for c in cores], dtype=np.int32)
        data = _f64(np.concatenate([_f64(c).reshape(-1) for c in cores]))
        return cls(lib.oc_mps_from_cores(d, _ip(ranks), _dp(data)))

    def cores(self) -> list[np.ndarray]:
        lib = _load()
        d = lib.oc_mps_sites(self.h)
        ranks = np.zeros(d + 1, dtype=np.int32)
        lib.oc_mps_ranks(self.h, _ip(ranks))
        sizes = [int(ranks[k]) * 2 * int(ranks[k + 1]) for k in range(d)]
        data = np.zeros(sum(sizes))
        lib.oc_mps_data(self.h, _dp(data))
        out, off = [], 0
        for k in range(d):
            out.append(data[off:off + sizes[k]].reshape(int(ranks[k]), 2, int(ranks[k + 1])).copy())
            off += sizes[k]
        return out


class _Mpo:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        if self.h:
            _load().oc_mpo_free(self.h)
            self.h = None

    def cores(self) -> list[np.ndarray]:
        lib = _load()
        d = lib.oc_mpo_sites(self.h)
        bonds = np.zeros(d + 1, dtype=np.int32)
        lib.oc_mpo_bonds(self.h, _ip(bonds))
        sizes = [int(bonds[k]) * 4 * int(bonds[k + 1]) for k in range(d)]
        data = np.zeros(sum(sizes))
        lib.oc_mpo_data(self.h, _dp(data))
        out, off = [], 0
        for k in range(d):
            out.append(data[off:off + sizes[k]].reshape(int(bonds[k]), 2, 2, int(bonds[k + 1])).copy())
            off += sizes[k]
        return out


# ---------------------------------------------------------------------------
# the oracle's calls, in the numpy oracle's formats
# ---------------------------------------------------------------------------
def svd(M: np.ndarray):
    """(U, S, Vt, sweeps) of the one-sided Jacobi SVD; sweeps = -1 if it hit its limit."""
    M = _f64(M)
    m, n = M.shape
    p = min(m, n)
    U, S, Vt = np.zeros((m, p)), np.zeros(p), np.zeros((p, n))
    sweeps = _load().oc_svd(m, n, _dp(M), _dp(U), _dp(S), _dp(Vt))
    return U, S, Vt, sweeps


def qr(A: np.ndarray):
    A = _f64(A)
    m, n = A.shape
    k = min(m, n)
    Q, R = np.zeros((m, k)), np.zeros((k, n))
    _load().oc_qr(m, n, _dp(A), _dp(Q), _dp(R))
    return Q, R


def trunc_rank(sigma, eps: float, chi: int) -> int:
    s = _f64(sigma)
    return int(_load().oc_trunc_rank(s.size, _dp(s), float(eps), int(chi)))


def mps_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    u = _f64(u)
    return _Mps(_load().oc_mps_from_dense(n, _ORDER[order], _dp(u), float(eps), int(chi))).cores()


def velocity_mps(c: np.ndarray, n: int, order: str, eps_c: float, chi_c: int) -> list[np.ndarray]:
    c = _f64(c)
    return mps_from_dense(c * c, n, order, eps_c, chi_c)


def mps_to_dense(cores: list[np.ndarray], n: int, order: str) -> np.ndarray:
    N = 1 << n
    out = np.zeros((N, N))
    A = _Mps.of(cores)
    _load().oc_mps_to_dense(A.h, n, _ORDER[order], _dp(out))
    return out


def mps_sample(cores: list[np.ndarray], n: int, order: str, ix, iz) -> np.ndarray:
    ix = np.ascontiguousarray(np.atleast_1d(ix), dtype=np.int32)
    iz = np.ascontiguousarray(np.atleast_1d(iz), dtype=np.int32)
    out = np.zeros(ix.size)
    A = _Mps.of(cores)
    _load().oc_mps_sample(A.h, n, _ORDER[order], ix.size, _ip(ix), _ip(iz), _dp(out))
    return out


def product_state(ix: int, iz: int, n: int, order: str) -> list[np.ndarray]:
    return _Mps(_load().oc_product_state(n, _ORDER[order], int(ix), int(iz))).cores()


def tt_round(cores: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    A = _Mps.of(cores)
    return _Mps(_load().oc_round(A.h, float(eps), int(chi))).cores()


def mps_sum(terms: list[tuple[float, list[np.ndarray]]]) -> list[np.ndarray]:
    hs = [_Mps.of(t[1]) for t in terms]
    coef = _f64([t[0] for t in terms])
    arr = (C.c_void_p * len(hs))(*[h.h for h in hs])
    return _Mps(_load().oc_sum(len(hs), _dp(coef), arr)).cores()


def shift_mpo_2d(n: int, axis: str, sign: int, bc: str, order: str) -> list[np.ndarray]:
    return _Mpo(_load().oc_shift_mpo(n, _AXIS[axis], int(sign), _BC[bc], _ORDER[order])).cores()


def laplacian_mpo(n: int, order: str, bc: str) -> list[np.ndarray]:
    return _Mpo(_load().oc_laplacian_mpo(n, _ORDER[order], _BC[bc])).cores()


def laplacian_sum_of_shifts(n: int, order: str, bc: str) -> list[np.ndarray]:
    return _Mpo(_load().oc_laplacian_sum_of_shifts(n, _ORDER[order], _BC[bc])).cores()


def _mpo_handle(kind: str, n: int, order: str, bc: str) -> _Mpo:
    lib = _load()
    f = lib.oc_laplacian_mpo if kind == "laplacian" else lib.oc_laplacian_sum_of_shifts
    return _Mpo(f(n, _ORDER[order], _BC[bc]))


def grid_operator(kind: str, n: int, order: str, bc: str, axis: str = "x", sign: int = 1) -> np.ndarray:
    """(N^2 x N^2) matrix of one of the oracle's MPOs acting on u flattened as
    x N + z: kind = 'laplacian' (five-state automaton), 'sum_of_shifts'
    (Eq. 16 as the plain bond-9 sum) or 'shift' (axis, sign)."""
    lib = _load()
    if kind == "shift":
        W = _Mpo(lib.oc_shift_mpo(n, _AXIS[axis], int(sign), _BC[bc], _ORDER[order]))
    else:
        W = _mpo_handle(kind, n, order, bc)
    NN = 1 << (2 * n)
    out = np.zeros((NN, NN))
    lib.oc_mpo_grid_operator(W.h, n, _ORDER[order], _dp(out))
    return out


def zipup_lr_laplacian(n: int, order: str, bc: str, A: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    """Zip-up of the oracle's own Laplacian MPO with A, sites 1 -> d."""
    W = _mpo_handle("laplacian", n, order, bc)
    B = _Mps.of(A)
    return _Mps(_load().oc_zipup_lr(W.h, B.h, float(eps), int(chi))).cores()


def zipup_rl_diagonal(c2: list[np.ndarray], A: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    """Zip-up of the diagonal MPO of c2 with A, sites d -> 1."""
    lib = _load()
    C2 = _Mps.of(c2)
    W = _Mpo(lib.oc_diagonal_mpo(C2.h))
    B = _Mps.of(A)
    return _Mps(lib.oc_zipup_rl(W.h, B.h, float(eps), int(chi))).cores()


def mps_step(n: int, order: str, bc: str, c2: list[np.ndarray], lambda2: float, prev: list[np.ndarray],
             cur: list[np.ndarray], eps: float, chi: int, src: tuple[int, int] | None = None,
             amp: float = 0.0) -> list[np.ndarray]:
    """One step of Eq. 17 with the oracle's own Laplacian MPO (Eq. 16)."""
    lib = _load()
    L = _mpo_handle("laplacian", n, order, bc)
    sx, sz = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    C2, P, Q = _Mps.of(c2), _Mps.of(prev), _Mps.of(cur)  # held until the call returns
    h = lib.oc_step(L.h, C2.h, float(lambda2), P.h, Q.h, float(eps), int(chi), sx, sz, float(amp), n,
                    _ORDER[order])
    return _Mps(h).cores()


def fdtd_step(u_prev: np.ndarray, u_cur: np.ndarray, c2: np.ndarray, lambda2: float, bc: str,
              src: tuple[int, int] | None = None, amp: float = 0.0) -> np.ndarray:
    u_prev, u_cur, c2 = _f64(u_prev), _f64(u_cur), _f64(c2)
    N = u_cur.shape[0]
    out = np.zeros((N, N))
    sx, sz = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    _load().oc_fdtd_step(N, _dp(u_prev), _dp(u_cur), _dp(c2), float(lambda2), _BC[bc], sx, sz, float(amp), _dp(out))
    return out


def mps_ranks(cores: list[np.ndarray]) -> list[int]:
    return [1] + [int(c.shape[2]) for c in cores]
