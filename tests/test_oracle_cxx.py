"""Pins for the C++ oracle (``oracle/qtt_oracle.cpp``), and the two oracles
against each other.

The C++ oracle is a second FP64 CPU implementation of the step, with its own
Householder QR and one-sided Jacobi SVD and no BLAS or LAPACK.  Pinned here
on its own, against what the paper and the mathematics fix:

* its factorisations: singular values prescribed by construction, orthonormal
  factors, A = Q R with R upper triangular and R^T R = A^T A, the zero and
  1 x 1 matrices, columns near the underflow threshold;
* the Sec. 4.3 truncation rule on hand-made spectra;
* (b) every shift MPO (Eq. 9-15) contracted to a matrix equals the
  brute-force permutation built from grid indices, and the Laplacian MPO
  (Eq. 16) equals the 5-point stencil, integer-exact, in its five-state form
  and as the plain bond-9 sum of shifts;
* (a) the untruncated MPS step (Eq. 17) equals the dense Eq. 2 update to
  1e-12, and its dense update equals a loop over grid points written here;
* (c) a discrete eigenmode follows its closed-form cosine recurrence (the
  periodic one to 1e-12 over 1000 steps);
* (d) separable fields have the closed-form QTT ranks;
* the leapfrog energy of the untruncated step is conserved;
* Eckart-Young on constructed spectra through the zip-up and the round;
* Eq. 7: the transition-operator MPO contracted to a matrix is
  2I + lambda^2 diag(c^2) times the 5-point stencil, and the untruncated
  fused step is Eq. 2;
* 3D (Sec. 6): the 7-point Laplacian MPO is the brute-force stencil, the
  untruncated 3D step is the dense 7-point update, separable fields have the
  product of their factors' ranks.

Then the two oracles are compared on truncated steps (2D, fused, 3D), where
neither is a plain definition: ranks equal and dense fields within 1e-10
relative L2."""
import math

import numpy as np
import pytest

from oracle import cxx as X
from oracle import qtt3d as Q3
from oracle import qtt_oracle as O
import workloads as W

ORDERS = ["sequential", "interleaved"]
BCS = ["periodic", "zero"]
INF = 1 << 30


# ---------------------------------------------------------------------------
# factorisations and the truncation rule
# ---------------------------------------------------------------------------
def _orth(m, k, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((m, k)))
    return Q


@pytest.mark.parametrize("m,n", [(1, 1), (1, 7), (7, 1), (6, 6), (40, 9), (9, 40), (64, 160), (33, 32)])
def test_jacobi_svd_recovers_prescribed_singular_values(m, n):
    rng = np.random.default_rng(m * 100 + n)
    p = min(m, n)
    s = np.sort(10.0 ** rng.uniform(-8, 1, p))[::-1]
    A = _orth(m, p, rng) @ np.diag(s) @ _orth(n, p, rng).T
    U, S, Vt, sweeps = X.svd(A)
    assert sweeps >= 0
    np.testing.assert_allclose(S, s, rtol=0, atol=2e-15 * max(m, n) * s[0])
    assert np.all(np.diff(S) <= 0.0)
    np.testing.assert_allclose(U.T @ U, np.eye(p), atol=1e-13)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(p), atol=1e-13)
    np.testing.assert_allclose(U @ np.diag(S) @ Vt, A, atol=1e-14 * max(m, n) * s[0])


def test_jacobi_svd_of_rank_deficient_and_zero_matrices():
    rng = np.random.default_rng(11)
    A = _orth(20, 3, rng) @ np.diag([5.0, 2.0, 1.0]) @ _orth(12, 3, rng).T
    U, S, Vt, sweeps = X.svd(A)
    assert sweeps >= 0
    np.testing.assert_allclose(S[:3], [5.0, 2.0, 1.0], atol=1e-13)
    assert np.all(np.abs(S[3:]) < 1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(12), atol=1e-12)  # completed to an orthonormal basis
    np.testing.assert_allclose(U @ np.diag(S) @ Vt, A, atol=1e-13)
    U, S, Vt, sweeps = X.svd(np.zeros((5, 3)))
    assert sweeps == 1 and np.all(S == 0.0)  # one sweep finds every pair orthogonal
    np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-15)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(3), atol=1e-15)
    U, S, Vt, _ = X.svd(np.array([[-3.0]]))
    assert S[0] == 3.0 and U[0, 0] * Vt[0, 0] == -1.0


@pytest.mark.parametrize("m,n", [(1, 1), (8, 3), (3, 8), (16, 16), (50, 20)])
def test_householder_qr_is_a_triangular_factorisation(m, n):
    rng = np.random.default_rng(7 * m + n)
    A = rng.standard_normal((m, n))
    Q, R = X.qr(A)
    k = min(m, n)
    assert Q.shape == (m, k) and R.shape == (k, n)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-14)
    assert np.all(np.tril(R, -1) == 0.0)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)
    np.testing.assert_allclose(R.T @ R, A.T @ A if m >= n else (Q @ R).T @ (Q @ R), atol=1e-12)


def test_householder_qr_of_dependent_and_zero_columns():
    A = np.zeros((6, 4))
    A[:, 1] = np.arange(6.0)
    A[:, 3] = 2.0 * A[:, 1]
    Q, R = X.qr(A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-14)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)


def test_factorisations_of_columns_near_the_underflow_threshold():
    """Columns of size 1e-160 .. 1e-300 next to columns of size 1: their
    squares underflow, so a reflector or a rotation built from unscaled
    sums of squares is not orthogonal.  Both factorisations stay orthogonal
    and reproduce the matrix to rounding (relative to its norm)."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((6, 9))
    A[:, 2] *= 1e-160
    A[:, 5] *= 1e-300
    A[3, :] *= 1e-170
    for M in (A, A.T):
        Q, R = X.qr(M)
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-14)
        assert np.linalg.norm(Q @ R - M) <= 1e-14 * np.linalg.norm(M)
        U, S, Vt, sweeps = X.svd(M)
        assert sweeps >= 0
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
        np.testing.assert_allclose(Vt @ Vt.T, np.eye(Vt.shape[0]), atol=1e-13)
        assert np.linalg.norm(U @ np.diag(S) @ Vt - M) <= 1e-14 * np.linalg.norm(M)
        np.testing.assert_allclose(S[:4], np.linalg.svd(M, compute_uv=False)[:4], rtol=1e-13)


@pytest.mark.parametrize("sc", [1e-10, 1e-100, 1e-160, 1e-200, 1e-300])
def test_jacobi_svd_resolves_a_tiny_column_to_relative_accuracy(sc):
    """[a, sc b]: sigma_1 = |a| and sigma_2 = sc |b - (a.b / a.a) a| up to a
    relative O(sc^2) (closed form of the 2-column case), which one-sided
    Jacobi reaches to rounding at any scale the exponent range holds."""
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(9), rng.standard_normal(9)
    U, S, Vt, sweeps = X.svd(np.stack([a, sc * b], axis=1))
    assert sweeps >= 0
    perp = b - (a @ b) / (a @ a) * a
    np.testing.assert_allclose(S, [np.linalg.norm(a), sc * np.linalg.norm(perp)], rtol=1e-14)
    assert abs(U[:, 0] @ U[:, 1]) < 1e-15


def test_trunc_rank_rule():
    s = np.array([4.0, 2.0, 1e-3, 4e-6, 3.9e-6, 0.0])
    assert X.trunc_rank(s, 1e-6, 100) == 4  # 4e-6 == eps * sigma_1 is kept
    assert X.trunc_rank(s, 1e-6, 2) == 2
    assert X.trunc_rank(s, 0.0, 100) == 6
    assert X.trunc_rank(np.zeros(5), 1e-6, 10) == 1
    assert X.trunc_rank(s, 0.9, 10) == 1


# ---------------------------------------------------------------------------
# (b) operators against brute force
# ---------------------------------------------------------------------------
def _shift_matrix(n, axis, sign, bc):
    N = 1 << n
    P = np.zeros((N * N, N * N))
    for x in range(N):
        for z in range(N):
            xx, zz = (x + sign, z) if axis == "x" else (x, z + sign)
            if bc == "periodic":
                xx, zz = xx % N, zz % N
            elif not (0 <= xx < N and 0 <= zz < N):
                continue
            P[xx * N + zz, x * N + z] = 1.0
    return P


def _stencil(n, bc):
    N = 1 << n
    B = np.zeros((N * N, N * N))
    for x in range(N):
        for z in range(N):
            i = x * N + z
            B[i, i] = -4.0
            for dx, dz in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, zz = x + dx, z + dz
                if bc == "periodic":
                    xx, zz = xx % N, zz % N
                elif not (0 <= xx < N and 0 <= zz < N):
                    continue
                B[i, xx * N + zz] += 1.0
    return B


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_shift_mpos_are_brute_force_shifts(n, order, bc):
    for axis in ("x", "z"):
        for sign in (+1, -1):
            got = X.grid_operator("shift", n, order, bc, axis, sign)
            np.testing.assert_array_equal(got, _shift_matrix(n, axis, sign, bc))


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_laplacian_mpo_is_the_five_point_stencil(n, order, bc):
    B = _stencil(n, bc)
    L = X.laplacian_mpo(n, order, bc)
    assert all(w.shape[0] <= 5 and w.shape[3] <= 5 for w in L)
    np.testing.assert_array_equal(X.grid_operator("laplacian", n, order, bc), B)
    if n <= 3:
        np.testing.assert_array_equal(X.grid_operator("sum_of_shifts", n, order, bc), B)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_laplacian_bonds_are_those_of_the_five_state_automaton(order, bc):
    """Bond 5 in the interior; states that cannot reach an accepted right
    boundary (zero boundary) or were never injected are removed."""
    n = 4
    bonds = [w.shape[3] for w in X.laplacian_mpo(n, order, bc)]
    assert bonds == [w.shape[3] for w in O.laplacian_mpo(n, order, bc)]
    assert bonds[-1] == 1 and max(bonds) == 5


# ---------------------------------------------------------------------------
# encoding and MPS algebra
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("order", ORDERS)
def test_tt_svd_round_trip_sample_and_left_orthonormal_cores(order):
    n = 4
    rng = np.random.default_rng(1)
    u = rng.standard_normal((16, 16))
    cores = X.mps_from_dense(u, n, order, 0.0, INF)
    assert np.linalg.norm(X.mps_to_dense(cores, n, order) - u) / np.linalg.norm(u) < 1e-14
    ix, iz = rng.integers(0, 16, 20), rng.integers(0, 16, 20)
    np.testing.assert_allclose(X.mps_sample(cores, n, order, ix, iz), u[ix, iz], rtol=1e-12, atol=1e-13)
    for c in cores[:-1]:
        M = c.reshape(-1, c.shape[2])
        np.testing.assert_allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
    # the site of each bit (Eq. 12 order): a point's one-hot state
    for (x, z) in ((5, 2), (15, 0), (0, 15)):
        ref = np.zeros((16, 16))
        ref[x, z] = 1.0
        np.testing.assert_array_equal(X.mps_to_dense(X.product_state(x, z, n, order), n, order), ref)


def test_mps_sum_is_the_dense_sum():
    rng = np.random.default_rng(2)
    n = 3
    u = [rng.standard_normal((8, 8)) for _ in range(3)]
    A = [X.mps_from_dense(v, n, "interleaved", 0.0, INF) for v in u]
    S = X.mps_sum([(2.0, A[0]), (-0.5, A[1]), (3.0, A[2])])
    np.testing.assert_allclose(X.mps_to_dense(S, n, "interleaved"), 2 * u[0] - 0.5 * u[1] + 3 * u[2], atol=1e-12)
    assert X.mps_ranks(S)[1:-1] == [a + b + c for a, b, c in zip(*(X.mps_ranks(t)[1:-1] for t in A))]


def test_round_truncates_to_prescribed_schmidt_values():
    """A 4 x 4 field u = Lf diag(2, 0.1) Rf^T in the sequential order (sites
    x_0, x_1, z_0, z_1): the middle bond carries the Schmidt values (2, 0.1)
    by construction.  Rounding the doubled state with eps = 0.1 discards
    0.1 < 0.1 * 2 and leaves the leading term (Eckart-Young); eps = 0.04
    keeps both."""
    rng = np.random.default_rng(4)
    Lf, Rf = _orth(4, 2, rng), _orth(4, 2, rng)
    s = np.array([2.0, 0.1])
    u = Lf @ np.diag(s) @ Rf.T
    A = X.mps_from_dense(u, 2, "sequential", 0.0, INF)
    B = X.tt_round(X.mps_sum([(0.5, A), (0.5, A)]), 0.1, 10)
    assert X.mps_ranks(B)[2] == 1
    np.testing.assert_allclose(X.mps_to_dense(B, 2, "sequential"), s[0] * np.outer(Lf[:, 0], Rf[:, 0]), atol=1e-12)
    B = X.tt_round(X.mps_sum([(0.5, A), (0.5, A)]), 0.04, 10)
    assert X.mps_ranks(B)[2] == 2
    np.testing.assert_allclose(X.mps_to_dense(B, 2, "sequential"), u, atol=1e-12)
    # right-orthonormal cores 2..d after the right-to-left sweep
    for c in B[1:]:
        M = c.reshape(c.shape[0], -1)
        np.testing.assert_allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-13)


def test_zipup_is_the_best_rank_r_approximation_on_two_sites():
    """d = 2 with the identity operator: the zip-up's single SVD sees the
    whole matrix, whose singular values are (3, 1e-3) by construction."""
    rng = np.random.default_rng(3)
    U, V = _orth(2, 2, rng), _orth(2, 2, rng)
    s = np.array([3.0, 1e-3])
    M = U @ np.diag(s) @ V.T
    # u[x, z] with n = 1: site 1 = x bit, site 2 = z bit in both orders
    ones = X.mps_from_dense(np.ones((2, 2)), 1, "sequential", 1e-12, INF)  # diag(1): the identity
    A = X.mps_from_dense(M, 1, "sequential", 0.0, INF)  # site 1 left-orthonormal
    out = X.zipup_rl_diagonal(ones, A, 1e-2, 10)
    np.testing.assert_allclose(X.mps_to_dense(out, 1, "sequential"), s[0] * np.outer(U[:, 0], V[:, 0]), atol=1e-14)
    out = X.zipup_rl_diagonal(ones, A, 1e-4, 10)
    np.testing.assert_allclose(X.mps_to_dense(out, 1, "sequential"), M, atol=1e-14)


# ---------------------------------------------------------------------------
# (a) the untruncated step is Eq. 2; (c) eigenmode; (d) separable ranks
# ---------------------------------------------------------------------------
def _fdtd_loops(up, uc, c2, lam2, bc, src, amp):
    N = uc.shape[0]

    def at(x, z):
        if bc == "periodic":
            return uc[x % N, z % N]
        return uc[x, z] if 0 <= x < N and 0 <= z < N else 0.0

    out = np.zeros_like(uc)
    for x in range(N):
        for z in range(N):
            lap = at(x + 1, z) + at(x - 1, z) + at(x, z + 1) + at(x, z - 1) - 4.0 * uc[x, z]
            out[x, z] = 2.0 * uc[x, z] - up[x, z] + lam2 * c2[x, z] * lap
    if src is not None:
        out[src] += amp
    return out


@pytest.mark.parametrize("bc", BCS)
def test_dense_update_is_eq2_written_as_loops(bc):
    rng = np.random.default_rng(9)
    up, uc = rng.standard_normal((8, 8)), rng.standard_normal((8, 8))
    c2 = rng.uniform(1.0, 4.0, (8, 8))
    np.testing.assert_allclose(X.fdtd_step(up, uc, c2, 0.1, bc, (3, 5), 0.7),
                               _fdtd_loops(up, uc, c2, 0.1, bc, (3, 5), 0.7), rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_untruncated_mps_step_equals_the_dense_update(order, bc):
    """Table 1: Eq. 17 in MPS form with chi = inf, eps = 0 is Eq. 2."""
    n = 3
    rng = np.random.default_rng(7)
    c = rng.uniform(1500.0, 3000.0, (8, 8))
    lam2 = (0.5 / c.max()) ** 2
    C = X.velocity_mps(c, n, order, 0.0, INF)
    c2 = X.mps_to_dense(C, n, order)
    np.testing.assert_allclose(c2, c * c, rtol=1e-13)
    zero = X.mps_from_dense(np.zeros((8, 8)), n, order, 0.0, INF)
    prev, cur = zero, zero
    up, uc = np.zeros((8, 8)), np.zeros((8, 8))
    src = (3, 5)
    for k in range(25):
        amp = math.sin(0.3 * k) + 0.1 * k
        nxt = X.mps_step(n, order, bc, C, lam2, prev, cur, 0.0, INF, src, amp)
        un = X.fdtd_step(up, uc, c2, lam2, bc, src, amp)
        prev, cur, up, uc = cur, nxt, uc, un
    got = X.mps_to_dense(cur, n, order)
    assert np.linalg.norm(got - uc) / np.linalg.norm(uc) < 1e-12


def _mode(n, p, q, bc):
    N = 1 << n
    x = np.arange(N)
    if bc == "periodic":
        fx, fz = np.cos(2 * np.pi * p * x / N), np.cos(2 * np.pi * q * x / N)
        mu = -4 * math.sin(math.pi * p / N) ** 2 - 4 * math.sin(math.pi * q / N) ** 2
    else:
        fx, fz = np.sin(np.pi * p * (x + 1) / (N + 1)), np.sin(np.pi * q * (x + 1) / (N + 1))
        mu = (2 * math.cos(math.pi * p / (N + 1)) - 2) + (2 * math.cos(math.pi * q / (N + 1)) - 2)
    return np.outer(fx, fz), mu


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("order", ORDERS)
def test_eigenmode_follows_the_cosine_recurrence(bc, order):
    """Constant c = 1, lambda^2 = 1/4: with u^0 the mode (eigenvalue mu of the
    5-point operator) and u^{-1} = cos(theta) u^0, cos(theta) = 1 +
    lambda^2 mu / 2, the scheme gives u^k = cos(k theta) u^0 exactly."""
    n = 5
    u0, mu = _mode(n, 1, 2, bc)
    lam2 = 0.25
    ct = 1.0 + lam2 * mu / 2.0
    th = math.acos(ct)
    C = X.velocity_mps(np.ones((32, 32)), n, order, 1e-14, 8)
    cur = X.mps_from_dense(u0, n, order, 1e-14, 8)
    prev = X.mps_from_dense(ct * u0, n, order, 1e-14, 8)
    for _ in range(300):
        prev, cur = cur, X.mps_step(n, order, bc, C, lam2, prev, cur, 1e-11, 16)
        assert max(X.mps_ranks(cur)) <= 4
    np.testing.assert_allclose(X.mps_to_dense(cur, n, order), math.cos(300 * th) * u0, atol=5e-12)


@pytest.mark.parametrize("order", ORDERS)
def test_periodic_eigenmode_over_1000_steps(order):
    """Check (c) at its full length: the periodic mode cos(2 pi x / N)
    cos(4 pi z / N) follows cos(k theta) to 1e-12 (relative L2) at every
    50th of 1000 steps, with no bond above rank 4."""
    n = 5
    u0, mu = _mode(n, 1, 2, "periodic")
    lam2 = 0.25
    ct = 1.0 + lam2 * mu / 2.0
    th = math.acos(ct)
    C = X.velocity_mps(np.ones((32, 32)), n, order, 1e-14, 8)
    cur = X.mps_from_dense(u0, n, order, 1e-14, 8)
    prev = X.mps_from_dense(ct * u0, n, order, 1e-14, 8)
    for k in range(1, 1001):
        prev, cur = cur, X.mps_step(n, order, "periodic", C, lam2, prev, cur, 1e-11, 16)
        assert max(X.mps_ranks(cur)) <= 4
        if k % 50 == 0:
            err = np.linalg.norm(X.mps_to_dense(cur, n, order) - math.cos(k * th) * u0) / np.linalg.norm(u0)
            assert err < 1e-12, (k, err)


@pytest.mark.parametrize("order", ORDERS)
def test_separable_fields_have_closed_form_ranks(order):
    """f(x) g(z): exp is rank 1 across every cut of its register, cos rank 2,
    a quadratic rank min(3, 2^m, 2^(n-m)), a delta rank 1; the cuts of the
    two registers multiply (interleaved) or follow each other (sequential)."""
    n = 5
    N = 1 << n
    x = np.arange(N, dtype=float)
    fams = {
        "exp": (np.exp(0.07 * x), lambda m: 1),
        "cos": (np.cos(0.3 * x + 0.2), lambda m: 1 if m in (0, n) else 2),
        "poly2": (1 + 0.5 * (x / N) - 2 * (x / N) ** 2, lambda m: min(3, 2 ** m, 2 ** (n - m))),
        "delta": ((x == 9).astype(float), lambda m: 1),
    }
    for fa, (f, rf) in fams.items():
        for ga, (g, rg) in fams.items():
            ranks = X.mps_ranks(X.mps_from_dense(np.outer(f, g), n, order, 1e-12, INF))
            if order == "sequential":
                exp = [1] + [rf(k) for k in range(1, n)] + [1] + [rg(k) for k in range(1, n)] + [1]
            else:
                exp = [1]
                for lev in range(n):
                    exp.append(rf(lev + 1) * rg(lev))
                    exp.append(rf(lev + 1) * rg(lev + 1))
                exp[-1] = 1
            assert ranks == exp, (fa, ga, ranks, exp)


@pytest.mark.parametrize("bc", BCS)
def test_leapfrog_energy_is_conserved_by_the_untruncated_step(bc):
    """Source-free, untruncated, variable c: the discrete energy of the Eq. 2
    leapfrog, sum (u^{k+1} - u^k)^2 / c^2 - lambda^2 <u^{k+1}, L u^k>, is
    constant to rounding for the symmetric 5-point L of either boundary."""
    n, order = 3, "interleaved"
    rng = np.random.default_rng(8)
    c = rng.uniform(1.0, 2.0, (8, 8))
    lam2 = 0.45 / (c * c).max()
    C = X.velocity_mps(c, n, order, 0.0, INF)
    c2 = X.mps_to_dense(C, n, order)
    B = _stencil(n, bc)

    def energy(u0, u1):
        return float(np.sum((u1 - u0) ** 2 / c2) - lam2 * np.dot(u1.reshape(-1), B @ u0.reshape(-1)))

    u_prev, u_cur = rng.standard_normal((8, 8)), rng.standard_normal((8, 8))
    prev, cur = X.mps_from_dense(u_prev, n, order, 0.0, INF), X.mps_from_dense(u_cur, n, order, 0.0, INF)
    E0 = energy(u_prev, u_cur)
    for _ in range(40):
        prev, cur = cur, X.mps_step(n, order, bc, C, lam2, prev, cur, 0.0, INF)
    E = energy(X.mps_to_dense(prev, n, order), X.mps_to_dense(cur, n, order))
    assert abs(E - E0) < 1e-11 * abs(E0)


# ---------------------------------------------------------------------------
# the transition operator of Eq. 7 and the 3D extension (Sec. 6)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_transition_operator_is_the_dense_eq7_operator(n, order, bc):
    """The MPO of A = 2I + lambda^2 C^2 L contracted to a matrix equals
    2I + lambda^2 diag(c^2) times the brute-force 5-point stencil."""
    N = 1 << n
    rng = np.random.default_rng(n * 10 + len(order) + len(bc))
    c = rng.uniform(1500.0, 3000.0, (N, N))
    lam2 = (0.5 / c.max()) ** 2
    C = X.velocity_mps(c, n, order, 0.0, INF)
    c2 = X.mps_to_dense(C, n, order)
    want = 2.0 * np.eye(N * N) + lam2 * c2.reshape(-1)[:, None] * _stencil(n, bc)
    got = X.a_operator_grid(n, order, bc, C, lam2)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    rc = X.mps_ranks(C)
    w = [1] + [W_.shape[3] for W_ in X.laplacian_mpo(n, order, bc)]
    assert X.a_operator_bonds(n, order, bc, C, lam2)[1:-1] == [a * b + 1 for a, b in zip(rc[1:-1], w[1:-1])]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_untruncated_fused_step_equals_the_dense_update(order, bc):
    """Eq. 7 in one zip-up with chi = inf, eps = 0 is Eq. 2.  Tolerance: one
    fused step from a random state is within 1e-14 of Eq. 2 (measured 7e-15;
    the Jacobi SVD's backward error grows with the rotations each column of
    the bond r_c w + 1 matrices takes), and the leapfrog carries an error
    injected at step j into every later step, so after k steps the errors add
    up to at most k^2 / 2 of one step's: 3.1e-12 at k = 25 (measured
    1.1e-12 .. 1.3e-12)."""
    n = 3
    rng = np.random.default_rng(17)
    c = rng.uniform(1500.0, 3000.0, (8, 8))
    lam2 = (0.5 / c.max()) ** 2
    C = X.velocity_mps(c, n, order, 0.0, INF)
    c2 = X.mps_to_dense(C, n, order)
    zero = X.mps_from_dense(np.zeros((8, 8)), n, order, 0.0, INF)
    prev, cur = zero, zero
    up, uc = np.zeros((8, 8)), np.zeros((8, 8))
    for k in range(25):
        amp = math.cos(0.2 * k) + 0.05 * k
        prev, cur = cur, X.mps_step_fused(n, order, bc, C, lam2, prev, cur, 0.0, INF, (2, 6), amp)
        up, uc = uc, X.fdtd_step(up, uc, c2, lam2, bc, (2, 6), amp)
    assert np.linalg.norm(X.mps_to_dense(cur, n, order) - uc) / np.linalg.norm(uc) < 0.5 * 25 ** 2 * 1e-14
    # one step from a random state
    u0, u1 = rng.standard_normal((8, 8)), rng.standard_normal((8, 8))
    P, Q = X.mps_from_dense(u0, n, order, 0.0, INF), X.mps_from_dense(u1, n, order, 0.0, INF)
    want = X.fdtd_step(u0, u1, c2, lam2, bc)
    got = X.mps_to_dense(X.mps_step_fused(n, order, bc, C, lam2, P, Q, 0.0, INF), n, order)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-14


def test_truncated_fused_step_agrees_with_the_numpy_oracle():
    n, chi, eps, order, bc = 5, 16, 1e-7, "interleaved", "periodic"
    N = 1 << n
    c = W.layered_model(n, 40.0, 12)
    lam2 = (0.5 / c.max()) ** 2
    prev = O.tt_round(W.random_tt_cores(2 * n, chi, 4, decay=0.1), 1e-14, chi)
    cur = O.tt_round(W.random_tt_cores(2 * n, chi, 5, decay=0.1), 1e-14, chi)
    A = O.a_operator_mpo(O.laplacian_mpo(n, order, bc), O.velocity_mps(c, n, order, 1e-8, 12), lam2)
    want = O.mps_step_fused(A, prev, cur, eps, chi, (N // 2 + 1, 3), 0.37, n, order)
    got = X.mps_step_fused(n, order, bc, X.velocity_mps(c, n, order, 1e-8, 12), lam2, prev, cur, eps, chi,
                           (N // 2 + 1, 3), 0.37)
    assert X.mps_ranks(got) == O.mps_ranks(want)
    ref = O.mps_to_dense(want, n, order)
    assert np.linalg.norm(X.mps_to_dense(got, n, order) - ref) / np.linalg.norm(ref) < 1e-10


def _stencil3(n, bc):
    N = 1 << n
    P = N ** 3
    B = np.zeros((P, P))
    for x in range(N):
        for y in range(N):
            for z in range(N):
                i = (x * N + y) * N + z
                B[i, i] = -6.0
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    q = [x + dx, y + dy, z + dz]
                    if bc == "periodic":
                        q = [v % N for v in q]
                    elif not all(0 <= v < N for v in q):
                        continue
                    B[i, (q[0] * N + q[1]) * N + q[2]] += 1.0
    return B


@pytest.mark.parametrize("n", [1, 2])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_3d_laplacian_is_the_seven_point_stencil(n, order, bc):
    B = _stencil3(n, bc)
    L = X.laplacian_mpo(n, order, bc, dims=3)
    assert all(w.shape[0] <= 7 and w.shape[3] <= 7 for w in L)
    np.testing.assert_array_equal(X.grid_operator("laplacian", n, order, bc, dims=3), B)
    np.testing.assert_array_equal(X.grid_operator("sum_of_shifts", n, order, bc, dims=3), B)
    if n == 2:
        assert [w.shape[3] for w in L] == [w.shape[3] for w in Q3.laplacian_mpo(n, order, bc)]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_untruncated_3d_step_equals_the_dense_seven_point_update(order, bc):
    n = 2
    rng = np.random.default_rng(23)
    c = rng.uniform(1500.0, 3000.0, (4, 4, 4))
    lam2 = 0.3 / c.max() ** 2
    C = X.velocity_mps(c, n, order, 0.0, INF)
    c2 = X.mps_to_dense(C, n, order, dims=3)
    np.testing.assert_allclose(c2, c * c, rtol=1e-13)
    zero = X.mps_from_dense(np.zeros((4, 4, 4)), n, order, 0.0, INF)
    prev, cur = zero, zero
    up, uc = np.zeros((4, 4, 4)), np.zeros((4, 4, 4))
    for k in range(20):
        amp = math.sin(0.4 * k) + 0.1 * k
        prev, cur = cur, X.mps_step(n, order, bc, C, lam2, prev, cur, 0.0, INF, (1, 2, 3), amp, dims=3)
        up, uc = uc, X.fdtd_step(up, uc, c2, lam2, bc, (1, 2, 3), amp)
    assert np.linalg.norm(X.mps_to_dense(cur, n, order, dims=3) - uc) / np.linalg.norm(uc) < 1e-12
    # the dense 7-point update is its stencil matrix
    u0, u1 = rng.standard_normal((4, 4, 4)), rng.standard_normal((4, 4, 4))
    want = 2 * u1 - u0 + lam2 * c2 * (_stencil3(n, bc) @ u1.reshape(-1)).reshape(4, 4, 4)
    np.testing.assert_allclose(X.fdtd_step(u0, u1, c2, lam2, bc), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("order", ORDERS)
def test_3d_separable_fields_have_the_product_of_their_factor_ranks(order):
    """f(x) g(y) h(z): the rank at a cut is the product of each factor's QTT
    rank at the split of its own register (exp: 1, cos: 2 inside the register,
    a quadratic: min(3, 2^m, 2^(n-m)))."""
    n = 3
    N = 1 << n
    x = np.arange(N, dtype=float)
    f, rf = np.cos(0.4 * x + 0.3), (lambda m: 1 if m in (0, n) else 2)
    g, rg = np.exp(0.1 * x), (lambda m: 1)
    h, rh = 1 + 0.5 * (x / N) - 2 * (x / N) ** 2, (lambda m: min(3, 2 ** m, 2 ** (n - m)))
    u = f[:, None, None] * g[None, :, None] * h[None, None, :]
    ranks = X.mps_ranks(X.mps_from_dense(u, n, order, 1e-12, INF))
    axes = Q3.site_axes(n, order)
    want = [1]
    seen = {"x": 0, "y": 0, "z": 0}
    for a, _b in axes:
        seen[a] += 1
        want.append(rf(seen["x"]) * rg(seen["y"]) * rh(seen["z"]))
    want[-1] = 1
    assert ranks == want


def test_3d_truncated_step_agrees_with_the_numpy_oracle():
    n, chi, eps, order, bc = 3, 12, 1e-6, "interleaved", "periodic"
    d = 3 * n
    rng = np.random.default_rng(31)
    c = rng.uniform(1500.0, 2500.0, (8, 8, 8))
    lam2 = 0.3 / c.max() ** 2
    prev = O.tt_round(W.random_tt_cores(d, chi, 6, decay=0.15), 1e-14, chi)
    cur = O.tt_round(W.random_tt_cores(d, chi, 7, decay=0.15), 1e-14, chi)
    want = Q3.mps_step(Q3.laplacian_mpo(n, order, bc), Q3.velocity_mps(c, n, order, 1e-8, 8), lam2, prev, cur,
                       eps, chi, (3, 4, 5), 0.2, n, order)
    got = X.mps_step(n, order, bc, X.velocity_mps(c, n, order, 1e-8, 8), lam2, prev, cur, eps, chi, (3, 4, 5), 0.2,
                     dims=3)
    assert X.mps_ranks(got) == O.mps_ranks(want)
    ref = Q3.mps_to_dense(want, n, order)
    assert np.linalg.norm(X.mps_to_dense(got, n, order, dims=3) - ref) / np.linalg.norm(ref) < 1e-10
    pts = [(0, 0, 0), (7, 3, 1), (3, 4, 5)]
    np.testing.assert_allclose(X.mps_sample_points(got, n, order, pts), ref[tuple(np.array(pts).T)], atol=1e-12)


# ---------------------------------------------------------------------------
# the two oracles against each other on truncated steps
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("seed", [1, 2])
def test_truncated_step_agrees_with_the_numpy_oracle(order, bc, seed):
    n, chi, eps = 5, 16, 1e-7
    N = 1 << n
    c = W.layered_model(n, 40.0, 10 + seed)
    lam2 = (0.5 / c.max()) ** 2
    prev = O.tt_round(W.random_tt_cores(2 * n, chi, 2 * seed, decay=0.1), 1e-14, chi)
    cur = O.tt_round(W.random_tt_cores(2 * n, chi, 2 * seed + 1, decay=0.1), 1e-14, chi)
    src, amp = (N // 2 + 1, 3), 0.37
    want = O.mps_step(O.laplacian_mpo(n, order, bc), O.velocity_mps(c, n, order, 1e-8, 12), lam2, prev, cur,
                      eps, chi, src, amp, n, order)
    Cx = X.velocity_mps(c, n, order, 1e-8, 12)
    assert X.mps_ranks(Cx) == O.mps_ranks(O.velocity_mps(c, n, order, 1e-8, 12))
    got = X.mps_step(n, order, bc, Cx, lam2, prev, cur, eps, chi, src, amp)
    assert X.mps_ranks(got) == O.mps_ranks(want)
    ref = O.mps_to_dense(want, n, order)
    assert np.linalg.norm(X.mps_to_dense(got, n, order) - ref) / np.linalg.norm(ref) < 1e-10


def test_zipups_and_round_agree_with_the_numpy_oracle():
    n, chi, eps, order, bc = 4, 12, 1e-6, "interleaved", "periodic"
    c = W.layered_model(n, 40.0, 5)
    A = O.tt_round(W.random_tt_cores(2 * n, chi, 9, decay=0.2), 1e-14, chi)
    phi_o = O.zipup_lr(O.laplacian_mpo(n, order, bc), A, eps, chi)
    phi_x = X.zipup_lr_laplacian(n, order, bc, A, eps, chi)
    assert X.mps_ranks(phi_x) == O.mps_ranks(phi_o)
    ref = O.mps_to_dense(phi_o, n, order)
    assert np.linalg.norm(X.mps_to_dense(phi_x, n, order) - ref) / np.linalg.norm(ref) < 1e-11
    C = O.velocity_mps(c, n, order, 1e-8, 10)
    eta_o = O.zipup_rl(O.diagonal_mpo(C), phi_o, eps, chi)
    eta_x = X.zipup_rl_diagonal(C, phi_o, eps, chi)
    assert X.mps_ranks(eta_x) == O.mps_ranks(eta_o)
    ref = O.mps_to_dense(eta_o, n, order)
    assert np.linalg.norm(X.mps_to_dense(eta_x, n, order) - ref) / np.linalg.norm(ref) < 1e-11
    th = O.mps_sum([(2.0, A), (-1.0, phi_o), (0.3, eta_o)])
    r_o, r_x = O.tt_round(th, eps, chi), X.tt_round(th, eps, chi)
    assert X.mps_ranks(r_x) == O.mps_ranks(r_o)
    ref = O.mps_to_dense(r_o, n, order)
    assert np.linalg.norm(X.mps_to_dense(r_x, n, order) - ref) / np.linalg.norm(ref) < 1e-11


def test_free_run_before_the_cap_binds_agrees_with_the_numpy_oracle():
    """40 steps of the 32 x 32 layered run from rest with a Ricker source,
    chi = 32 (not reached), eps = 1e-8: the two oracles stay within 1e-9."""
    n, chi, eps, order, bc = 5, 32, 1e-8, "interleaved", "periodic"
    N = 1 << n
    c = W.layered_model(n, 20.0, 3)
    dh = 20.0
    dt = 0.5 * dh / c.max()
    lam2 = (dt / dh) ** 2
    L = O.laplacian_mpo(n, order, bc)
    Co, Cx = O.velocity_mps(c, n, order, 1e-8, 16), X.velocity_mps(c, n, order, 1e-8, 16)
    zero = O.zero_mps(2 * n)
    po, co, px, cx = zero, zero, zero, zero
    src = (N // 2, 2)
    for k in range(40):
        amp = lam2 * float(W.ricker(k * dt - 1.5 / 15.0, 15.0)) * 1e3
        po, co = co, O.mps_step(L, Co, lam2, po, co, eps, chi, src, amp, n, order)
        px, cx = cx, X.mps_step(n, order, bc, Cx, lam2, px, cx, eps, chi, src, amp)
    assert max(O.mps_ranks(co)) < chi
    ref = O.mps_to_dense(co, n, order)
    assert np.linalg.norm(X.mps_to_dense(cx, n, order) - ref) / np.linalg.norm(ref) < 1e-9


# ---------------------------------------------------------------------------
# independence of the oracles and the library
# ---------------------------------------------------------------------------
def test_oracles_and_library_share_no_code():
    """The C++ oracle includes only standard headers; neither oracle imports
    the package; the package loads nothing from the oracles."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "qtt_oracle.cpp")).read()
    incs = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert incs and all(re.fullmatch(r"[a-z_]+", h) for h in incs), incs
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith(".py"):
            assert "paper_2609_01904_b300" not in open(os.path.join(root, "oracle", f)).read(), f
    pkg = os.path.join(root, "paper_2609_01904_b300")
    for dirpath, _dirs, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b|qtt_oracle|oracle/", text, re.M), f


@pytest.mark.parametrize("order", ORDERS)
def test_step_at_a_binding_cap_agrees_with_the_numpy_oracle(order):
    """The regime of the long runs: every interior bond at the cap chi = 32
    on a 64 x 64 layered section; ranks equal, fields within 1e-10."""
    n, chi, eps, bc = 6, 32, 1e-6, "periodic"
    c = W.layered_model(n, 20.0, 3)
    lam2 = (0.5 / c.max()) ** 2
    prev = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.05), 1e-14, chi)
    cur = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.05), 1e-14, chi)
    want = O.mps_step(O.laplacian_mpo(n, order, bc), O.velocity_mps(c, n, order, 1e-8, chi), lam2, prev, cur,
                      eps, chi)
    got = X.mps_step(n, order, bc, X.velocity_mps(c, n, order, 1e-8, chi), lam2, prev, cur, eps, chi)
    assert max(O.mps_ranks(want)) == chi
    assert X.mps_ranks(got) == O.mps_ranks(want)
    ref = O.mps_to_dense(want, n, order)
    assert np.linalg.norm(X.mps_to_dense(got, n, order) - ref) / np.linalg.norm(ref) < 1e-10
