"""FP64 CPU oracle for the MPS (quantized tensor-train) wave-equation step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library: it is written from the paper's equations with
plain numpy, using ``numpy.linalg.svd`` / ``numpy.linalg.qr`` / ``numpy.einsum``
as library primitives and no blocking, fusion or reordering beyond what the
method states.

Paper: "Quantum Circuit and Tensor Network Implementation of the 2D Acoustic
Wave Equation" (Nemeth & Vattay).

Conventions (readings of the paper are listed where they are used):

* grid u[x, z], N = 2^n per axis, x horizontal, z depth (Sec. 2, Eq. 2);
* d = 2n binary sites in the tensor-product order of Eq. 12 (W^[0] first),
  i.e. least significant bit first, bit m being x_m of Eq. 3; SEQUENTIAL
  puts the x register before the z register (Eq. 14-15); INTERLEAVED
  alternates x_0, z_0, x_1, z_1, ...;
* MPS core k has shape [r_{k-1}][2][r_k] (Eq. 8), boundary bonds r_0 = r_d = 1;
* MPO core k has shape [w_l][t (out)][s (in)][w_r];
* truncation keeps sigma_i >= eps * sigma_1, then caps at chi, keeps >= 1
  (Sec. 4.3: values with lambda_i < eps * lambda_max are discarded and the bond
  is capped at chi_max).

Every function below says which passage it follows.  Functions without an
independent pin say "parity unpinned" in their docstring; at the time of
writing every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import numpy as np

SEQUENTIAL = "sequential"
INTERLEAVED = "interleaved"
PERIODIC = "periodic"
ZERO = "zero"

# identity, raising (|1><0|) and lowering (|0><1|) operators, [out][in]
_I = np.eye(2)
_SP = np.array([[0.0, 0.0], [1.0, 0.0]])  # sigma^+ = |1><0|
_SM = np.array([[0.0, 1.0], [0.0, 0.0]])  # sigma^- = |0><1|
_X = _SP + _SM


# ---------------------------------------------------------------------------
# Register encoding (Sec. 3, Eq. 3; Sec. 4.2, Eq. 12, Eq. 14-15)
# ---------------------------------------------------------------------------
def site_axes(n: int, order: str) -> list[tuple[str, int]]:
    """(axis, bit) carried by each of the d = 2n sites.

    Sites follow the tensor-product order of Eq. 12, W^[0] (x) W^[1] (x) ...,
    i.e. the least significant bit first; bit m is x_m of Eq. 3.  SEQUENTIAL
    puts the x register before the z register (Eq. 14-15); INTERLEAVED
    alternates x_0, z_0, x_1, z_1, ..."""
    if order == SEQUENTIAL:
        return [("x", i) for i in range(n)] + [("z", i) for i in range(n)]
    if order == INTERLEAVED:
        out = []
        for i in range(n):
            out += [("x", i), ("z", i)]
        return out
    raise ValueError(order)


def site_bits(ix: int, iz: int, n: int, order: str) -> list[int]:
    """Binary digits s_1..s_d of grid point (ix, iz) (Eq. 3 basis state)."""
    return [((ix if ax == "x" else iz) >> b) & 1 for ax, b in site_axes(n, order)]


def _perm(n: int, order: str) -> list[int]:
    # axis of u.reshape((2,)*2n): x bit b -> n-1-b, z bit b -> 2n-1-b
    return [(n - 1 - b) if ax == "x" else (2 * n - 1 - b) for ax, b in site_axes(n, order)]


def dense_to_tensor(u: np.ndarray, n: int, order: str) -> np.ndarray:
    """u[x, z] -> order-d tensor indexed by (s_1, ..., s_d) (Eq. 3)."""
    t = np.asarray(u, dtype=np.float64).reshape((2,) * (2 * n))
    return np.transpose(t, _perm(n, order))


def tensor_to_dense(t: np.ndarray, n: int, order: str) -> np.ndarray:
    """Inverse of :func:`dense_to_tensor`."""
    N = 1 << n
    inv = np.argsort(_perm(n, order))
    return np.transpose(np.asarray(t).reshape((2,) * (2 * n)), inv).reshape(N, N)


# ---------------------------------------------------------------------------
# Truncation rule (Sec. 4.3)
# ---------------------------------------------------------------------------
def trunc_rank(sigma: np.ndarray, eps: float, chi: int) -> int:
    """Number of singular values kept (Sec. 4.3): discard sigma_i < eps*sigma_1,
    cap at chi, keep at least one (an all-zero matrix keeps rank 1)."""
    s = np.asarray(sigma, dtype=np.float64)
    if s.size == 0 or s[0] == 0.0:
        return 1
    r = int(np.count_nonzero(s >= eps * s[0]))
    return max(1, min(r, int(chi)))


def discarded_weight(sigma: np.ndarray, r: int) -> float:
    """Sum of squares of the discarded singular values."""
    s = np.asarray(sigma, dtype=np.float64)
    return float(np.sum(s[r:] ** 2))


def _svd(M: np.ndarray):
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    return U, S, Vt


# ---------------------------------------------------------------------------
# MPS construction and readout (Sec. 4.1, Eq. 8)
# ---------------------------------------------------------------------------
def tt_svd(t: np.ndarray, eps: float, chi: int, stats: list | None = None) -> list[np.ndarray]:
    """Sequential left-to-right SVDs of the reshaped tensor (Eq. 8), each bond
    truncated by :func:`trunc_rank`.  Cores 1..d-1 are left-orthonormal."""
    d = t.ndim
    cores = []
    r = 1
    M = np.asarray(t, dtype=np.float64).reshape(1, -1)
    for k in range(d - 1):
        M = M.reshape(r * 2, -1)
        U, S, Vt = _svd(M)
        rk = trunc_rank(S, eps, chi)
        if stats is not None:
            stats.append((k + 1, S.copy(), rk))
        cores.append(U[:, :rk].reshape(r, 2, rk))
        M = S[:rk, None] * Vt[:rk]
        r = rk
    cores.append(M.reshape(r, 2, 1))
    return cores


def mps_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    """TT-SVD of a dense field u[x, z] (Eq. 3 then Eq. 8)."""
    return tt_svd(dense_to_tensor(u, n, order), eps, chi)


def state_from_dense(u: np.ndarray, n: int, order: str, eps: float, chi: int) -> list[np.ndarray]:
    """A state for the stepper: TT-SVD (Eq. 8), then the Sec. 4.3 compression,
    which leaves cores 2..d right-orthonormal (the zip-up of Eq. 16 sweeps
    from site 1 and measures the truncation in that gauge)."""
    return tt_round(mps_from_dense(u, n, order, eps, chi), eps, chi)


def velocity_mps(c: np.ndarray, n: int, order: str, eps_c: float, chi_c: int) -> list[np.ndarray]:
    """MPS of the squared velocity c^2(x, z) (Eq. 4), by TT-SVD (Eq. 8)."""
    c = np.asarray(c, dtype=np.float64)
    return mps_from_dense(c * c, n, order, eps_c, chi_c)


def mps_full(cores: list[np.ndarray]) -> np.ndarray:
    """Contract all cores into the order-d tensor (Eq. 8, summed over bonds)."""
    out = cores[0]  # [1][2][r1]
    for c in cores[1:]:
        out = np.tensordot(out, c, axes=([-1], [0]))
    return out.reshape((2,) * len(cores))


def mps_to_dense(cores: list[np.ndarray], n: int, order: str) -> np.ndarray:
    return tensor_to_dense(mps_full(cores), n, order)


def mps_sample(cores: list[np.ndarray], n: int, order: str, ix, iz) -> np.ndarray:
    """u(x, z) = A^(1)_{s_1} ... A^(d)_{s_d} (Eq. 8) for each requested point."""
    ix = np.atleast_1d(ix)
    iz = np.atleast_1d(iz)
    out = np.empty(ix.shape[0])
    for p in range(ix.shape[0]):
        bits = site_bits(int(ix[p]), int(iz[p]), n, order)
        v = np.ones((1,))
        for c, s in zip(cores, bits):
            v = v @ c[:, s, :]
        out[p] = v[0]
    return out


def mps_ranks(cores: list[np.ndarray]) -> list[int]:
    return [1] + [int(c.shape[2]) for c in cores]


def zero_mps(d: int) -> list[np.ndarray]:
    """Rank-1 MPS of the zero field."""
    return [np.zeros((1, 2, 1)) for _ in range(d)]


def product_state(ix: int, iz: int, n: int, order: str) -> list[np.ndarray]:
    """Rank-1 MPS of the unit impulse at (ix, iz): one-hot cores of its bits."""
    cores = []
    for s in site_bits(ix, iz, n, order):
        c = np.zeros((1, 2, 1))
        c[0, s, 0] = 1.0
        cores.append(c)
    return cores


# ---------------------------------------------------------------------------
# Shift operators (Sec. 3.1 Eq. 5, Fig. 1; Sec. 4.2 Eq. 9-15)
# ---------------------------------------------------------------------------
def incrementer_circuit(x: int, n: int) -> int:
    """Gate-level incrementer of Fig. 1 / Eq. 5: from the MSB down to the LSB,
    bit m is flipped when all less significant bits are 1."""
    bits = [(x >> m) & 1 for m in range(n)]
    for m in range(n - 1, -1, -1):
        ctrl = 1
        for l in range(m):
            ctrl &= bits[l]
        bits[m] ^= ctrl
    return sum(b << m for m, b in enumerate(bits))


def shift_mpo_1d(n: int, sign: int, bc: str, literal_eq11: bool = False) -> list[np.ndarray]:
    """1D shift MPO S^+ (sign=+1, Eq. 9-12) or S^- (sign=-1, Eq. 13) on n
    sites, least significant bit first (Eq. 12).  The bond is the carry: core
    m is core[alpha_{m-1}][t][s][alpha_m] = W^[m][alpha_{m-1}][alpha_m] (Eq. 9:
    row = incoming carry, column = outgoing carry).

    W^[0] injects carry 1 (Eq. 10).  At the most significant bit the outgoing
    carry is summed over for the periodic wrap-around the text states
    (Sec. 3.1, Sec. 4.2), or only carry 0 is kept, which is the terminal
    tensor Eq. 11 prints (``literal_eq11`` or bc == 'zero'): that shift drops
    the overflow, so it is the shift with zeros outside the grid."""
    hit, miss = (_SP, _SM) if sign > 0 else (_SM, _SP)
    bulk = np.zeros((2, 2, 2, 2))  # [a_in][t][s][a_out]  (Eq. 9 / Eq. 13)
    bulk[0, :, :, 0] = _I
    bulk[1, :, :, 0] = hit
    bulk[1, :, :, 1] = miss
    cores = []
    for m in range(n):
        core = bulk.copy()
        if m == 0:  # Eq. 10: carry 1 injected at the LSB
            core = core[1:2]
        if m == n - 1:  # terminal, Eq. 11 or its periodic counterpart
            keep_overflow = (bc == PERIODIC) and not literal_eq11
            w = np.array([1.0, 1.0 if keep_overflow else 0.0])
            core = np.tensordot(core, w, axes=([3], [0]))[..., None]
        cores.append(core)
    return cores


def identity_mpo(n: int) -> list[np.ndarray]:
    return [np.eye(2).reshape(1, 2, 2, 1) for _ in range(n)]


def shift_mpo_2d(n: int, axis: str, sign: int, bc: str, order: str) -> list[np.ndarray]:
    """S_x^{+-} = S^{+-} (x) I and S_z^{+-} = I (x) S^{+-} (Eq. 14-15) in the
    chosen site order.  In the interleaved order the carry passes through the
    other axis' sites on identity cores."""
    one = iter(shift_mpo_1d(n, sign, bc))
    out = []
    carry_dim = 1
    for ax, _b in site_axes(n, order):  # left to right, with the carry
        if ax == axis:
            c = next(one)
            carry_dim = c.shape[3]
        else:
            c = np.einsum("ab,ts->atsb", np.eye(carry_dim), _I)
        out.append(c)
    return out


# ---------------------------------------------------------------------------
# Laplacian MPO (Sec. 3.1 Eq. 6, Sec. 4.3 Eq. 16)
# ---------------------------------------------------------------------------
# Bond states of the Laplacian automaton, shared by the whole sum of Eq. 16.
# The bond to the right of a site says what the less significant bits (to its
# left) have done: D = no pending carry (identity from here on), XP/XM = S_x^+/-
# with a carry/borrow still pending, ZP/ZM likewise for z.
_D, _XP, _XM, _ZP, _ZM = range(5)


def laplacian_mpo(n: int, order: str, bc: str) -> list[np.ndarray]:
    """MPO of S_x^+ + S_x^- + S_z^+ + S_z^- - 4I (Eq. 16), written as one
    carry automaton with five bond states instead of a bond-9 sum of MPOs.

    Left boundary (before the least significant site): weight -4 on D and 1
    on each of XP, XM, ZP, ZM (each shift injects its carry, Eq. 10).  Site
    of axis a, core[left][t][s][right]: D->D by I; AP->AP by sigma^- (bit
    1 -> 0, carry moves on); AP->D by sigma^+ (bit 0 -> 1, carry absorbed);
    AM->AM by sigma^+; AM->D by sigma^-; the other axis' states pass through
    by I (Eq. 9 and Eq. 13 with the carry on the bond).  Right boundary:
    periodic accepts every state (the overflow wraps, Sec. 3.1); zero accepts
    only D (the overflow is dropped, as Eq. 11 prints).

    Bond states that are zero on either side are removed, so the bond is 5 in
    the interior of the interleaved order."""
    d = 2 * n
    W = []
    for ax, _b in site_axes(n, order):
        w = np.zeros((5, 2, 2, 5))  # [left][t][s][right]
        w[_D, :, :, _D] = _I
        p, m = (_XP, _XM) if ax == "x" else (_ZP, _ZM)
        op, om = (_ZP, _ZM) if ax == "x" else (_XP, _XM)
        w[p, :, :, p] = _SM
        w[p, :, :, _D] = _SP
        w[m, :, :, m] = _SP
        w[m, :, :, _D] = _SM
        w[op, :, :, op] = _I
        w[om, :, :, om] = _I
        W.append(w)
    inject = np.array([-4.0, 1.0, 1.0, 1.0, 1.0])
    accept = np.ones(5) if bc == PERIODIC else np.array([1.0, 0.0, 0.0, 0.0, 0.0])
    W[0] = np.tensordot(inject, W[0], axes=([0], [0]))[None]
    W[-1] = np.tensordot(W[-1], accept, axes=([3], [0]))[..., None]
    # drop bond states that are zero on either side (exact: removes zero slices),
    # repeated until no bond shrinks
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


def mpo_to_dense(W: list[np.ndarray]) -> np.ndarray:
    """Operator matrix in the site basis: out index (t_1..t_d), in (s_1..s_d)."""
    d = len(W)
    T = W[0][0]  # [t][s][w]
    T = T.reshape(2, 2, -1)
    outs, ins = 2, 2
    for k in range(1, d):
        T = np.einsum("abw,wtsv->atbsv", T.reshape(outs, ins, -1), W[k])
        outs *= 2
        ins *= 2
        T = T.reshape(outs, ins, -1)
    return T[:, :, 0]


def line_operator(W: list[np.ndarray], n: int) -> np.ndarray:
    """1D MPO as an (N x N) matrix acting on a vector indexed by x, with site
    m carrying bit m of x (Eq. 12 order)."""
    M = mpo_to_dense(W)
    idx = np.array([int(np.ravel_multi_index(tuple((x >> m) & 1 for m in range(n)), (2,) * n))
                    for x in range(1 << n)])
    return M[np.ix_(idx, idx)]


def grid_operator(W: list[np.ndarray], n: int, order: str) -> np.ndarray:
    """MPO as an (N^2 x N^2) matrix acting on u flattened as x*N + z."""
    N = 1 << n
    M = mpo_to_dense(W)
    idx = np.array([[int(np.ravel_multi_index(tuple(site_bits(x, z, n, order)), (2,) * (2 * n)))
                     for z in range(N)] for x in range(N)]).reshape(-1)
    return M[np.ix_(idx, idx)]


# ---------------------------------------------------------------------------
# MPS algebra (Sec. 4.3, Eq. 17 and the compression paragraph)
# ---------------------------------------------------------------------------
def diagonal_mpo(cores: list[np.ndarray]) -> list[np.ndarray]:
    """Diagonal MPO of an MPS (Sec. 4.3: C^2 as a diagonal MPO):
    W[r][t][s][r'] = delta_{ts} B[r][s][r']."""
    out = []
    for B in cores:
        W = np.zeros((B.shape[0], 2, 2, B.shape[2]))
        W[:, 0, 0, :] = B[:, 0, :]
        W[:, 1, 1, :] = B[:, 1, :]
        out.append(W)
    return out


def zipup_lr(W: list[np.ndarray], A: list[np.ndarray], eps: float, chi: int,
             stats: list | None = None) -> list[np.ndarray]:
    """MPO x MPS by zip-up from site 1 to site d, truncating at every bond.

    At site k the carried tensor C[a][w][b] (new bond, MPO bond, MPS bond) is
    contracted with the MPS core and the MPO core,
        T[a][t][w'][b'] = sum_{w,s,b} C[a][w][b] A_k[b][s][b'] W_k[w][t][s][w'],
    the matrix T[(a,t)][(w',b')] is split by an SVD, U becomes output core k
    (truncated by the Sec. 4.3 rule) and S V^T is carried to site k+1."""
    d = len(A)
    C = np.ones((1, 1, 1))
    out = []
    for k in range(d):
        T = np.einsum("awb,bsc,wtsv->atvc", C, A[k], W[k], optimize=True)
        a, _t, wv, bc = T.shape
        M = T.reshape(a * 2, wv * bc)
        if k == d - 1:
            out.append(M.reshape(a, 2, 1))
            break
        U, S, Vt = _svd(M)
        r = trunc_rank(S, eps, chi)
        if stats is not None:
            stats.append(("zip_lr", k + 1, S.copy(), r))
        out.append(U[:, :r].reshape(a, 2, r))
        C = (S[:r, None] * Vt[:r]).reshape(r, wv, bc)
    return out


def zipup_rl(W: list[np.ndarray], A: list[np.ndarray], eps: float, chi: int,
             stats: list | None = None) -> list[np.ndarray]:
    """Mirror of :func:`zipup_lr`, sweeping from site d to site 1:
        T[b][w][t][a'] = sum_{s,b',w'} A_k[b][s][b'] W_k[w][t][s][w'] C[b'][w'][a'],
    the matrix T[(b,w)][(t,a')] is split by an SVD, V^T becomes output core k
    and U S is carried to site k-1."""
    d = len(A)
    C = np.ones((1, 1, 1))
    out: list = [None] * d
    for k in range(d - 1, -1, -1):
        T = np.einsum("bsc,wtsv,cva->bwta", A[k], W[k], C, optimize=True)
        b, w, _t, a = T.shape
        M = T.reshape(b * w, 2 * a)
        if k == 0:
            out[0] = M.reshape(1, 2, a)
            break
        U, S, Vt = _svd(M)
        r = trunc_rank(S, eps, chi)
        if stats is not None:
            stats.append(("zip_rl", k, S.copy(), r))
        out[k] = Vt[:r].reshape(r, 2, a)
        C = (U[:, :r] * S[:r]).reshape(b, w, r)
    return out


def mps_sum(terms: list[tuple[float, list[np.ndarray]]]) -> list[np.ndarray]:
    """sum_j c_j |psi_j> as one MPS (Sec. 4.3): the first cores are placed side
    by side with the coefficients folded in, the middle cores block-diagonally
    and the last cores stacked, so bonds add up."""
    d = len(terms[0][1])
    out = []
    for k in range(d):
        blocks = [t[1][k] for t in terms]
        L = 1 if k == 0 else sum(b.shape[0] for b in blocks)
        R = 1 if k == d - 1 else sum(b.shape[2] for b in blocks)
        core = np.zeros((L, 2, R))
        lo = ro = 0
        for (coef, _), b in zip(terms, blocks):
            l, _, r = b.shape
            if k == 0:
                core[:, :, ro:ro + r] += coef * b
            elif k == d - 1:
                core[lo:lo + l, :, :] += b
            else:
                core[lo:lo + l, :, ro:ro + r] = b
            lo += l if k > 0 else 0
            ro += r if k < d - 1 else 0
        out.append(core)
    return out


def tt_round(A: list[np.ndarray], eps: float, chi: int, stats: list | None = None) -> list[np.ndarray]:
    """Compression (Sec. 4.3): a left-to-right QR orthogonalisation sweep,
    then a right-to-left SVD sweep truncating each bond by the Sec. 4.3 rule."""
    A = [np.array(c, dtype=np.float64) for c in A]
    d = len(A)
    for k in range(d - 1):
        l, _, r = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(l * 2, r))
        A[k] = Q.reshape(l, 2, Q.shape[1])
        A[k + 1] = np.einsum("ij,jsk->isk", R, A[k + 1])
    for k in range(d - 1, 0, -1):
        l, _, r = A[k].shape
        U, S, Vt = _svd(A[k].reshape(l, 2 * r))
        rr = trunc_rank(S, eps, chi)
        if stats is not None:
            stats.append(("round", k, S.copy(), rr))
        A[k] = Vt[:rr].reshape(rr, 2, r)
        A[k - 1] = np.einsum("isj,jk->isk", A[k - 1], U[:, :rr] * S[:rr])
    return A


def mps_step(L: list[np.ndarray], c2: list[np.ndarray], lambda2: float,
             prev: list[np.ndarray], cur: list[np.ndarray], eps: float, chi: int,
             src: tuple[int, int] | None = None, amp: float = 0.0,
             n: int | None = None, order: str | None = None,
             stats: list | None = None) -> list[np.ndarray]:
    """One time step of Eq. 17 in MPS form:
        phi   = L psi^k                  (zip-up, sites 1 -> d)
        eta   = C^2 phi                  (zip-up with diag(c^2), sites d -> 1)
        theta = 2 psi^k - psi^{k-1} + lambda^2 eta [+ amp * e_src]
        psi^{k+1} = round(theta)         (QR sweep 1 -> d, SVD sweep d -> 1).
    Returns psi^{k+1}."""
    phi = zipup_lr(L, cur, eps, chi, stats)
    eta = zipup_rl(diagonal_mpo(c2), phi, eps, chi, stats)
    terms = [(2.0, cur), (-1.0, prev), (lambda2, eta)]
    if src is not None:
        terms.append((amp, product_state(src[0], src[1], n, order)))
    theta = mps_sum(terms)
    return tt_round(theta, eps, chi, stats)


# ---------------------------------------------------------------------------
# Fused transition operator (Eq. 7): A = 2I + lambda^2 C^2 L
# ---------------------------------------------------------------------------
def mpo_product(W_out: list[np.ndarray], W_in: list[np.ndarray]) -> list[np.ndarray]:
    """MPO of the operator product W_out W_in (W_in acts first): core k is
    sum_u W_out[a][t][u][a'] W_in[b][u][s][b'] on the bond pairs (a, b)."""
    out = []
    for A, B in zip(W_out, W_in):
        P = np.einsum("atub,cusd->actsbd", A, B)
        out.append(P.reshape(A.shape[0] * B.shape[0], 2, 2, A.shape[3] * B.shape[3]))
    return out


def mpo_sum(terms: list[tuple[float, list[np.ndarray]]]) -> list[np.ndarray]:
    """sum_j c_j W_j as one MPO, built like :func:`mps_sum`: first cores side
    by side with the coefficients, middle cores block-diagonal, last cores
    stacked."""
    d = len(terms[0][1])
    out = []
    for k in range(d):
        blocks = [t[1][k] for t in terms]
        L = 1 if k == 0 else sum(b.shape[0] for b in blocks)
        R = 1 if k == d - 1 else sum(b.shape[3] for b in blocks)
        core = np.zeros((L, 2, 2, R))
        lo = ro = 0
        for (coef, _), b in zip(terms, blocks):
            l, _, _, r = b.shape
            if k == 0:
                core[:, :, :, ro:ro + r] += coef * b
            elif k == d - 1:
                core[lo:lo + l] += b
            else:
                core[lo:lo + l, :, :, ro:ro + r] = b
            lo += l if k > 0 else 0
            ro += r if k < d - 1 else 0
        out.append(core)
    return out


def a_operator_mpo(L: list[np.ndarray], c2: list[np.ndarray], lambda2: float) -> list[np.ndarray]:
    """MPO of the transition operator of Eq. 7, A = 2I + lambda^2 C^2 L: the
    diagonal MPO of c^2 (Sec. 4.3) times the Laplacian MPO (Eq. 16), plus
    twice the identity; bond r_c w + 1.

    Balancing (a reading: the paper gives no representation of A): the c^2
    MPS keeps its whole norm (~c_max^2, 1e6..1e7 m^2/s^2) in its last core, so
    the product term would be ~lambda^2 ~ 1e-8 against the identity's 1 at
    every bond the zip-up cuts, and FP64 rounding of the cut would be
    amplified by the last core.  The norm nu of the last c^2 core is moved
    into the coefficient: lambda^2 nu on the first core, the last c^2 core
    divided by nu.  The operator is unchanged."""
    d = len(L)
    B = [np.array(x, dtype=np.float64) for x in c2]
    nu = float(np.linalg.norm(B[-1]))
    if nu > 0.0:
        B[-1] = B[-1] / nu
    else:
        nu = 1.0
    return mpo_sum([(lambda2 * nu, mpo_product(diagonal_mpo(B), L)), (2.0, [np.eye(2).reshape(1, 2, 2, 1)] * d)])


def mps_step_fused(A: list[np.ndarray], prev: list[np.ndarray], cur: list[np.ndarray], eps: float, chi: int,
                   src: tuple[int, int] | None = None, amp: float = 0.0, n: int | None = None,
                   order: str | None = None, stats: list | None = None) -> list[np.ndarray]:
    """The step of Eq. 7 with A applied as one operator:
        phi       = A psi^k                 (zip-up of A, sites 1 -> d)
        theta     = phi - psi^{k-1} [+ amp * e_src]
        psi^{k+1} = round(theta).
    In exact arithmetic this is the step of :func:`mps_step`; the truncation
    points differ (one zip-up instead of two)."""
    phi = zipup_lr(A, cur, eps, chi, stats)
    terms = [(1.0, phi), (-1.0, prev)]
    if src is not None:
        terms.append((amp, product_state(src[0], src[1], n, order)))
    return tt_round(mps_sum(terms), eps, chi, stats)


# ---------------------------------------------------------------------------
# Dense FDTD (Sec. 2, Eq. 2)
# ---------------------------------------------------------------------------
def neighbour_sum(u: np.ndarray, bc: str) -> np.ndarray:
    """u_{i+1,j} + u_{i-1,j} + u_{i,j+1} + u_{i,j-1} with the boundary rule:
    periodic wrap, or zero outside the grid."""
    if bc == PERIODIC:
        return (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1))
    p = np.zeros((u.shape[0] + 2, u.shape[1] + 2))
    p[1:-1, 1:-1] = u
    return p[2:, 1:-1] + p[:-2, 1:-1] + p[1:-1, 2:] + p[1:-1, :-2]


def fdtd_step(u_prev: np.ndarray, u_cur: np.ndarray, c2: np.ndarray, lambda2: float,
              bc: str, src: tuple[int, int] | None = None, amp: float = 0.0) -> np.ndarray:
    """Eq. 2: u^{k+1} = 2u^k - u^{k-1} + lambda^2 c^2 (sum of 4 neighbours - 4u^k),
    plus amp at the source point."""
    nxt = 2.0 * u_cur - u_prev + lambda2 * c2 * (neighbour_sum(u_cur, bc) - 4.0 * u_cur)
    if src is not None:
        nxt[src[0], src[1]] += amp
    return nxt


def leapfrog_energy(u_cur: np.ndarray, u_nxt: np.ndarray, c2: np.ndarray, lambda2: float,
                    bc: str) -> float:
    """Discrete energy of the Eq. 2 scheme between levels k and k+1:
    sum (u^{k+1}-u^k)^2 / c^2 - lambda^2 <u^{k+1}, L u^k>, L the 5-point
    operator; conserved exactly (up to rounding) for a symmetric L."""
    Lu = neighbour_sum(u_cur, bc) - 4.0 * u_cur
    return float(np.sum((u_nxt - u_cur) ** 2 / c2) - lambda2 * np.sum(u_nxt * Lu))
