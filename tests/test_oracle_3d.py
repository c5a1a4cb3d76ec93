"""Pins of the 3D oracle (oracle/qtt3d.py) against what the mathematics fixes:
the 7-point stencil built by brute force from grid indices, the dense 3D
update of Eq. 2 (Table 1's identity with one more axis), the closed-form
ranks of separable fields, and the encoding round trip."""
import math

import numpy as np
import pytest

from oracle import qtt3d as O3
from oracle import qtt_oracle as O

ORDERS = ["sequential", "interleaved"]
BCS = ["periodic", "zero"]
INF = 1 << 30


def _stencil3(n, bc):
    N = 1 << n
    M = np.zeros((N ** 3, N ** 3))
    for x in range(N):
        for y in range(N):
            for z in range(N):
                i = (x * N + y) * N + z
                M[i, i] = -6.0
                for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if bc == "periodic":
                        M[i, ((xx % N) * N + yy % N) * N + zz % N] += 1.0
                    elif 0 <= xx < N and 0 <= yy < N and 0 <= zz < N:
                        M[i, (xx * N + yy) * N + zz] += 1.0
    return M


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [1, 2])
def test_3d_laplacian_mpo_is_the_seven_point_stencil(order, bc, n):
    W = O3.laplacian_mpo(n, order, bc)
    assert np.array_equal(O3.grid_operator(W, n, order), _stencil3(n, bc))
    if n == 2 and order == "interleaved":
        assert max(w.shape[3] for w in W[:-1]) == 7


@pytest.mark.parametrize("order", ORDERS)
def test_3d_encoding_round_trip_and_sampling(order):
    n = 2
    N = 1 << n
    rng = np.random.default_rng(1)
    u = rng.standard_normal((N, N, N))
    t = O3.dense_to_tensor(u, n, order)
    assert np.array_equal(O3.tensor_to_dense(t, n, order), u)
    for p in ((0, 0, 0), (1, 2, 3), (3, 0, 2)):
        assert t[tuple(O3.site_bits(p, n, order))] == u[p]
    A = O3.mps_from_dense(u, n, order, 0.0, INF)
    pts = [(1, 2, 3), (3, 3, 0), (0, 1, 1)]
    np.testing.assert_allclose(O3.mps_sample(A, n, order, pts), [u[p] for p in pts], rtol=1e-12)
    d = O3.product_state((2, 1, 3), n, order)
    e = np.zeros((N, N, N))
    e[2, 1, 3] = 1.0
    assert np.array_equal(O3.mps_to_dense(d, n, order), e)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_untruncated_3d_mps_step_equals_the_dense_update(order, bc):
    """Table 1 in 3D: chi = inf, eps = 0 reproduces the 7-point Eq. 2 update."""
    n = 2
    N = 1 << n
    rng = np.random.default_rng(2)
    c = rng.uniform(1500.0, 3000.0, (N, N, N))
    lam2 = (0.4 / c.max()) ** 2
    C = O3.velocity_mps(c, n, order, 0.0, INF)
    c2r = O3.mps_to_dense(C, n, order)
    np.testing.assert_allclose(c2r, c * c, rtol=1e-13)
    L = O3.laplacian_mpo(n, order, bc)
    d = 3 * n
    prev, cur = O.zero_mps(d), O.zero_mps(d)
    up, uc = np.zeros((N, N, N)), np.zeros((N, N, N))
    src = (1, 2, 3)
    for k in range(20):
        amp = math.sin(0.3 * k) + 0.1 * k
        nxt = O3.mps_step(L, C, lam2, prev, cur, 0.0, INF, src, amp, n, order)
        un = O3.fdtd_step(up, uc, c2r, lam2, bc, src, amp)
        prev, cur = cur, nxt
        up, uc = uc, un
    assert np.linalg.norm(O3.mps_to_dense(cur, n, order) - uc) / np.linalg.norm(uc) < 1e-12


def test_3d_separable_field_ranks():
    """f(x) g(y) h(z) in the sequential order has rank 1 at the bonds between
    the axis registers; exponentials have QTT rank 1 and cosines rank 2 within
    a register."""
    n = 3
    N = 1 << n
    x = np.arange(N)
    f = np.exp(0.3 * x)
    g = np.cos(1.3 * x + 0.4)
    h = 1.0 + 0.5 * x
    u = f[:, None, None] * g[None, :, None] * h[None, None, :]
    A = O3.mps_from_dense(u, n, "sequential", 1e-12, INF)
    r = O.mps_ranks(A)
    assert r[n] == 1 and r[2 * n] == 1
    assert r[1:n] == [1] * (n - 1)            # exponential in x
    assert r[n + 1:2 * n] == [2] * (n - 1)    # cosine in y
    assert r[2 * n + 1:3 * n] == [2] * (n - 1)  # degree-1 polynomial in z
