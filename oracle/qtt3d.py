"""FP64 CPU oracle of the 3D extension of the MPS wave step (the paper's
discussion section states that 3D wavefields follow the same construction).

TEST INFRASTRUCTURE ONLY, like ``oracle.qtt_oracle`` (whose generic MPS
operations it reuses: TT-SVD, zip-ups, sums, the round and the truncation
rule of Sec. 4.3).  Nothing in the product path may import it.

The 2D construction carries over axis by axis:

* grid u[x, y, z], N = 2^n per axis, dense index (x N + y) N + z;
* d = 3n binary sites, least significant bit first per axis (Eq. 12 order);
  SEQUENTIAL: x_0..x_{n-1}, y_0..y_{n-1}, z_0..z_{n-1} (Eq. 14-15 with three
  registers); INTERLEAVED: x_0, y_0, z_0, x_1, y_1, z_1, ...;
* the 7-point Laplacian S_x^+ + S_x^- + S_y^+ + S_y^- + S_z^+ + S_z^- - 6I
  (Eq. 6 and Eq. 16 with a third pair of shifts), as one carry automaton of
  seven bond states (no carry pending; a carry or borrow pending for each of
  the six shifts), with the boundary rule of the 2D operator;
* the explicit update u^{k+1} = 2u^k - u^{k-1} + lambda^2 c^2 (L u^k) (Eq. 2
  with the 7-point stencil), the source as a rank-1 product state.

Every function is pinned by tests/test_oracle_3d.py (brute-force stencil,
untruncated step = dense update, separable ranks)."""
from __future__ import annotations

import numpy as np

from oracle import qtt_oracle as O

AXES = ("x", "y", "z")


def site_axes(n: int, order: str) -> list[tuple[str, int]]:
    """(axis, bit) carried by each of the d = 3n sites (least significant bit
    first per axis)."""
    if order == O.SEQUENTIAL:
        return [(a, i) for a in AXES for i in range(n)]
    if order == O.INTERLEAVED:
        return [(a, i) for i in range(n) for a in AXES]
    raise ValueError(order)


def site_bits(p: tuple[int, int, int], n: int, order: str) -> list[int]:
    """Binary digits s_1..s_d of grid point p = (ix, iy, iz)."""
    c = dict(zip(AXES, p))
    return [(c[a] >> b) & 1 for a, b in site_axes(n, order)]


def _perm(n: int, order: str) -> list[int]:
    # axis of u.reshape((2,)*3n): bit b of axis a sits at a * n + (n - 1 - b)
    return [AXES.index(a) * n + (n - 1 - b) for a, b in site_axes(n, order)]


def dense_to_tensor(u: np.ndarray, n: int, order: str) -> np.ndarray:
    t = np.asarray(u, dtype=np.float64).reshape((2,) * (3 * n))
    return np.transpose(t, _perm(n, order))


def tensor_to_dense(t: np.ndarray, n: int, order: str) -> np.ndarray:
    N = 1 << n
    inv = np.argsort(_perm(n, order))
    return np.transpose(np.asarray(t).reshape((2,) * (3 * n)), inv).reshape(N, N, N)


def mps_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    return O.tt_svd(dense_to_tensor(u, n, order), eps, chi)


def state_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    """TT-SVD (Eq. 8), then the Sec. 4.3 compression (right-orthonormal)."""
    return O.tt_round(mps_from_dense(u, n, order, eps, chi), eps, chi)


def velocity_mps(c: np.ndarray, n: int, order: str, eps_c: float, chi_c: int) -> list[np.ndarray]:
    """MPS of c^2 by TT-SVD (Eq. 4, Eq. 8)."""
    return mps_from_dense(c * c, n, order, eps_c, chi_c)


def mps_to_dense(cores: list[np.ndarray], n: int, order: str) -> np.ndarray:
    return tensor_to_dense(O.mps_full(cores), n, order)


def mps_sample(cores: list[np.ndarray], n: int, order: str, pts) -> np.ndarray:
    """u(p) = A^(1)_{s_1} ... A^(d)_{s_d} (Eq. 8) for each point p."""
    out = np.empty(len(pts))
    for i, p in enumerate(pts):
        v = np.ones((1,))
        for c, s in zip(cores, site_bits(tuple(int(x) for x in p), n, order)):
            v = v @ c[:, s, :]
        out[i] = v[0]
    return out


def product_state(p: tuple[int, int, int], n: int, order: str) -> list[np.ndarray]:
    """Rank-1 MPS of the unit impulse at p."""
    cores = []
    for s in site_bits(p, n, order):
        c = np.zeros((1, 2, 1))
        c[0, s, 0] = 1.0
        cores.append(c)
    return cores


# bond states of the automaton: no carry pending, then (+, -) per axis
_D = 0


def _states(axis: int) -> tuple[int, int]:
    return 1 + 2 * axis, 2 + 2 * axis


def laplacian_mpo(n: int, order: str, bc: str) -> list[np.ndarray]:
    """MPO of the 7-point Laplacian sum_a (S_a^+ + S_a^-) - 6I, one carry
    automaton with seven bond states.  Left boundary: -6 on D, 1 on each
    shift state (the carry of Eq. 10).  A site of axis a maps its own states
    as in Eq. 9 (S^+: carry moves on by sigma^-, is absorbed by sigma^+) and
    Eq. 13 (S^-: the reverse), passes the other axes' states through by I and
    keeps D by I.  Right boundary: periodic accepts every state, zero only D
    (Eq. 11 as printed).  States zero on either side of a bond are removed."""
    ns = 7
    W = []
    for ax, _b in site_axes(n, order):
        a = AXES.index(ax)
        w = np.zeros((ns, 2, 2, ns))
        w[_D, :, :, _D] = O._I
        for other in range(3):
            p, m = _states(other)
            if other == a:
                w[p, :, :, p] = O._SM
                w[p, :, :, _D] = O._SP
                w[m, :, :, m] = O._SP
                w[m, :, :, _D] = O._SM
            else:
                w[p, :, :, p] = O._I
                w[m, :, :, m] = O._I
        W.append(w)
    inject = np.array([-6.0] + [1.0] * 6)
    accept = np.ones(ns) if bc == O.PERIODIC else np.array([1.0] + [0.0] * 6)
    W[0] = np.tensordot(inject, W[0], axes=([0], [0]))[None]
    W[-1] = np.tensordot(W[-1], accept, axes=([3], [0]))[..., None]
    d = len(W)
    changed = True
    while changed:
        changed = False
        for k in range(d - 1):
            live_l = np.any(W[k] != 0.0, axis=(0, 1, 2))
            live_r = np.any(W[k + 1] != 0.0, axis=(1, 2, 3))
            keep = np.nonzero(live_l & live_r)[0]
            if keep.size < W[k].shape[3]:
                W[k] = W[k][..., keep]
                W[k + 1] = W[k + 1][keep]
                changed = True
    return W


def grid_operator(W: list[np.ndarray], n: int, order: str) -> np.ndarray:
    """MPO as an (N^3 x N^3) matrix acting on u flattened as (x N + y) N + z."""
    N = 1 << n
    M = O.mpo_to_dense(W)
    idx = np.array([int(np.ravel_multi_index(tuple(site_bits((x, y, z), n, order)), (2,) * (3 * n)))
                    for x in range(N) for y in range(N) for z in range(N)])
    return M[np.ix_(idx, idx)]


def mps_step(L, c2, lambda2, prev, cur, eps, chi, src=None, amp=0.0, n=None, order=None, stats=None):
    """The step of Eq. 17 in 3D: zip-up of L (sites 1 -> d), zip-up of
    diag(c^2) (d -> 1), the sum with the source, the round."""
    phi = O.zipup_lr(L, cur, eps, chi, stats)
    eta = O.zipup_rl(O.diagonal_mpo(c2), phi, eps, chi, stats)
    terms = [(2.0, cur), (-1.0, prev), (lambda2, eta)]
    if src is not None:
        terms.append((amp, product_state(src, n, order)))
    return O.tt_round(O.mps_sum(terms), eps, chi, stats)


def neighbour_sum(u: np.ndarray, bc: str) -> np.ndarray:
    """Sum of the six face neighbours: periodic wrap, or zero outside."""
    if bc == O.PERIODIC:
        return sum(np.roll(u, s, a) for a in range(3) for s in (1, -1))
    p = np.zeros(tuple(s + 2 for s in u.shape))
    p[1:-1, 1:-1, 1:-1] = u
    return (p[2:, 1:-1, 1:-1] + p[:-2, 1:-1, 1:-1] + p[1:-1, 2:, 1:-1] + p[1:-1, :-2, 1:-1] + p[1:-1, 1:-1, 2:]
            + p[1:-1, 1:-1, :-2])


def fdtd_step(u_prev, u_cur, c2, lambda2, bc, src=None, amp=0.0):
    """Eq. 2 with the 7-point stencil."""
    nxt = 2.0 * u_cur - u_prev + lambda2 * c2 * (neighbour_sum(u_cur, bc) - 6.0 * u_cur)
    if src is not None:
        nxt[src] += amp
    return nxt
