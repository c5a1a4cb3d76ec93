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
        "oc_mps_from_dense": (vp, [i, i, i, dp, d, i]),
        "oc_mps_to_dense": (None, [vp, i, i, i, dp]),
        "oc_mps_sample": (None, [vp, i, i, i, i, ip, dp]),
        "oc_product_state": (vp, [i, i, i, ip]),
        "oc_round": (vp, [vp, d, i]),
        "oc_sum": (vp, [i, dp, C.POINTER(vp)]),
        "oc_shift_mpo": (vp, [i, i, i, i, i, i]),
        "oc_laplacian_mpo": (vp, [i, i, i, i]),
        "oc_laplacian_sum_of_shifts": (vp, [i, i, i, i]),
        "oc_diagonal_mpo": (vp, [vp]),
        "oc_a_operator_mpo": (vp, [vp, vp, d]),
        "oc_mpo_sites": (i, [vp]),
        "oc_mpo_bonds": (None, [vp, ip]),
        "oc_mpo_data": (None, [vp, dp]),
        "oc_mpo_grid_operator": (None, [vp, i, i, i, dp]),
        "oc_mpo_free": (None, [vp]),
        "oc_zipup_lr": (vp, [vp, vp, d, i]),
        "oc_zipup_rl": (vp, [vp, vp, d, i]),
        "oc_step": (vp, [vp, vp, d, vp, vp, d, i, ip, d, i, i, i]),
        "oc_step_fused": (vp, [vp, vp, vp, d, i, ip, d, i, i, i]),
        "oc_fdtd_step": (None, [i, i, dp, dp, dp, d, i, ip, d, dp]),
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


def _dims(u) -> int:
    return 3 if np.ndim(u) == 3 else 2


def _pt(p) -> np.ndarray:
    return np.ascontiguousarray(p, dtype=np.int32)


def mps_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    """TT-SVD (Eq. 8) of a dense field u[x, z] or u[x, y, z]."""
    u = _f64(u)
    return _Mps(_load().oc_mps_from_dense(_dims(u), n, _ORDER[order], _dp(u), float(eps), int(chi))).cores()


def velocity_mps(c: np.ndarray, n: int, order: str, eps_c: float, chi_c: int) -> list[np.ndarray]:
    c = _f64(c)
    return mps_from_dense(c * c, n, order, eps_c, chi_c)


def mps_to_dense(cores: list[np.ndarray], n: int, order: str, dims: int = 2) -> np.ndarray:
    N = 1 << n
    out = np.zeros((N,) * dims)
    A = _Mps.of(cores)
    _load().oc_mps_to_dense(A.h, dims, n, _ORDER[order], _dp(out))
    return out


def mps_sample(cores: list[np.ndarray], n: int, order: str, ix, iz) -> np.ndarray:
    """u at the points (ix[p], iz[p]) of a 2D grid."""
    pts = np.stack([np.atleast_1d(ix), np.atleast_1d(iz)], axis=1)
    return mps_sample_points(cores, n, order, pts)


def mps_sample_points(cores: list[np.ndarray], n: int, order: str, pts) -> np.ndarray:
    """u at each point of pts (np x dims)."""
    pts = _pt(np.atleast_2d(pts))
    out = np.zeros(pts.shape[0])
    A = _Mps.of(cores)
    _load().oc_mps_sample(A.h, pts.shape[1], n, _ORDER[order], pts.shape[0], _ip(pts), _dp(out))
    return out


def product_state(ix: int, iz: int, n: int, order: str) -> list[np.ndarray]:
    return point_state((ix, iz), n, order)


def point_state(p, n: int, order: str) -> list[np.ndarray]:
    """Rank-1 MPS of the unit impulse at the point p (2 or 3 coordinates)."""
    p = _pt(p)
    return _Mps(_load().oc_product_state(p.size, n, _ORDER[order], _ip(p))).cores()


def tt_round(cores: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    A = _Mps.of(cores)
    return _Mps(_load().oc_round(A.h, float(eps), int(chi))).cores()


def mps_sum(terms: list[tuple[float, list[np.ndarray]]]) -> list[np.ndarray]:
    hs = [_Mps.of(t[1]) for t in terms]
    coef = _f64([t[0] for t in terms])
    arr = (C.c_void_p * len(hs))(*[h.h for h in hs])
    return _Mps(_load().oc_sum(len(hs), _dp(coef), arr)).cores()


def _laplacian(kind: str, n: int, order: str, bc: str, dims: int) -> _Mpo:
    lib = _load()
    f = lib.oc_laplacian_mpo if kind == "laplacian" else lib.oc_laplacian_sum_of_shifts
    return _Mpo(f(dims, n, _ORDER[order], _BC[bc]))


def laplacian_mpo(n: int, order: str, bc: str, dims: int = 2) -> list[np.ndarray]:
    return _laplacian("laplacian", n, order, bc, dims).cores()


def laplacian_sum_of_shifts(n: int, order: str, bc: str, dims: int = 2) -> list[np.ndarray]:
    return _laplacian("sum_of_shifts", n, order, bc, dims).cores()


def shift_mpo(n: int, axis: str, sign: int, bc: str, order: str, dims: int = 2) -> list[np.ndarray]:
    return _Mpo(_load().oc_shift_mpo(dims, n, _ORDER[order], _axis(axis, dims), int(sign), _BC[bc])).cores()


def _axis(axis: str, dims: int) -> int:
    return {"x": 0, "y": 1, "z": dims - 1}[axis]


def grid_operator(kind: str, n: int, order: str, bc: str, axis: str = "x", sign: int = 1,
                  dims: int = 2) -> np.ndarray:
    """(N^dims x N^dims) matrix of one of the oracle's MPOs acting on the
    dense field flattened in its layout: kind = 'laplacian' (the automaton),
    'sum_of_shifts' (Eq. 16 as the plain sum) or 'shift' (axis, sign)."""
    lib = _load()
    if kind == "shift":
        W = _Mpo(lib.oc_shift_mpo(dims, n, _ORDER[order], _axis(axis, dims), int(sign), _BC[bc]))
    else:
        W = _laplacian(kind, n, order, bc, dims)
    P = 1 << (dims * n)
    out = np.zeros((P, P))
    lib.oc_mpo_grid_operator(W.h, dims, n, _ORDER[order], _dp(out))
    return out


def a_operator_grid(n: int, order: str, bc: str, c2: list[np.ndarray], lambda2: float) -> np.ndarray:
    """(N^2 x N^2) matrix of the oracle's MPO of Eq. 7, A = 2I + lambda^2 C^2 L."""
    lib = _load()
    L = _laplacian("laplacian", n, order, bc, 2)
    C2 = _Mps.of(c2)
    A = _Mpo(lib.oc_a_operator_mpo(L.h, C2.h, float(lambda2)))
    P = 1 << (2 * n)
    out = np.zeros((P, P))
    lib.oc_mpo_grid_operator(A.h, 2, n, _ORDER[order], _dp(out))
    return out


def a_operator_bonds(n: int, order: str, bc: str, c2: list[np.ndarray], lambda2: float) -> list[int]:
    lib = _load()
    L = _laplacian("laplacian", n, order, bc, 2)
    C2 = _Mps.of(c2)
    A = _Mpo(lib.oc_a_operator_mpo(L.h, C2.h, float(lambda2)))
    return [1] + [int(w.shape[3]) for w in A.cores()]


def zipup_lr_laplacian(n: int, order: str, bc: str, A: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    """Zip-up of the oracle's own Laplacian MPO with A, sites 1 -> d."""
    W = _laplacian("laplacian", n, order, bc, 2)
    B = _Mps.of(A)
    return _Mps(_load().oc_zipup_lr(W.h, B.h, float(eps), int(chi))).cores()


def zipup_rl_diagonal(c2: list[np.ndarray], A: list[np.ndarray], eps: float, chi: int) -> list[np.ndarray]:
    """Zip-up of the diagonal MPO of c2 with A, sites d -> 1."""
    lib = _load()
    C2 = _Mps.of(c2)
    W = _Mpo(lib.oc_diagonal_mpo(C2.h))
    B = _Mps.of(A)
    return _Mps(lib.oc_zipup_rl(W.h, B.h, float(eps), int(chi))).cores()


def _src(src, dims):
    if src is None:
        return None, None
    p = _pt(src)
    assert p.size == dims
    return p, _ip(p)


def mps_step(n: int, order: str, bc: str, c2: list[np.ndarray], lambda2: float, prev: list[np.ndarray],
             cur: list[np.ndarray], eps: float, chi: int, src=None, amp: float = 0.0,
             dims: int = 2) -> list[np.ndarray]:
    """One step of Eq. 17 with the oracle's own Laplacian MPO (Eq. 16; the
    7-point operator when dims = 3)."""
    lib = _load()
    L = _laplacian("laplacian", n, order, bc, dims)
    C2, P, Q = _Mps.of(c2), _Mps.of(prev), _Mps.of(cur)  # held until the call returns
    keep, sp = _src(src, dims)
    h = lib.oc_step(L.h, C2.h, float(lambda2), P.h, Q.h, float(eps), int(chi), sp, float(amp), dims, n,
                    _ORDER[order])
    return _Mps(h).cores()


def mps_step_fused(n: int, order: str, bc: str, c2: list[np.ndarray], lambda2: float, prev: list[np.ndarray],
                   cur: list[np.ndarray], eps: float, chi: int, src=None, amp: float = 0.0) -> list[np.ndarray]:
    """The step of Eq. 7 with A = 2I + lambda^2 C^2 L applied as one MPO."""
    lib = _load()
    L = _laplacian("laplacian", n, order, bc, 2)
    C2, P, Q = _Mps.of(c2), _Mps.of(prev), _Mps.of(cur)
    A = _Mpo(lib.oc_a_operator_mpo(L.h, C2.h, float(lambda2)))
    keep, sp = _src(src, 2)
    h = lib.oc_step_fused(A.h, P.h, Q.h, float(eps), int(chi), sp, float(amp), 2, n, _ORDER[order])
    return _Mps(h).cores()


def fdtd_step(u_prev: np.ndarray, u_cur: np.ndarray, c2: np.ndarray, lambda2: float, bc: str,
              src=None, amp: float = 0.0) -> np.ndarray:
    """Eq. 2 (the 7-point stencil for a 3D field)."""
    u_prev, u_cur, c2 = _f64(u_prev), _f64(u_cur), _f64(c2)
    dims = _dims(u_cur)
    n = int(u_cur.shape[0]).bit_length() - 1
    out = np.zeros(u_cur.shape)
    keep, sp = _src(src, dims)
    _load().oc_fdtd_step(dims, n, _dp(u_prev), _dp(u_cur), _dp(c2), float(lambda2), _BC[bc], sp, float(amp),
                         _dp(out))
    return out


def mps_ranks(cores: list[np.ndarray]) -> list[int]:
    return [1] + [int(c.shape[2]) for c in cores]
