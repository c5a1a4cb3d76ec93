"""Pins for the oracle's encoding, shift and Laplacian MPOs.

Each check compares the oracle against something that is not the oracle: the
paper's printed circuit (Fig. 1) and tensors (Eq. 9-13), brute-force
permutation / stencil matrices built by explicit loops over the grid, and the
stated mappings |x> -> |(x +- 1) mod 2^n> (Sec. 3.1, Sec. 4.2)."""
import os

import numpy as np
import pytest

from oracle import qtt_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ORDERS = [O.SEQUENTIAL, O.INTERLEAVED]
BCS = [O.PERIODIC, O.ZERO]


def _read_fig1():
    gates, mapping = [], {}
    with open(os.path.join(GOLD, "fig1_incrementer.txt")) as f:
        for line in f:
            p = line.split("#")[0].split()
            if not p:
                continue
            if p[0] == "gate":
                gates.append((int(p[1]), [int(c) for c in p[2:]]))
            elif p[0] == "map":
                mapping[int(p[1])] = int(p[2])
    return gates, mapping


def test_fig1_circuit_matches_printed_mapping_and_oracle():
    gates, mapping = _read_fig1()
    for x in range(8):
        bits = [(x >> m) & 1 for m in range(3)]
        for tgt, ctrls in gates:  # multi-controlled X, in the printed order
            if all(bits[c] for c in ctrls):
                bits[tgt] ^= 1
        y = sum(b << m for m, b in enumerate(bits))
        assert y == mapping[x]
        assert O.incrementer_circuit(x, 3) == mapping[x]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_incrementer_circuit_is_cyclic_increment(n):
    for x in range(1 << n):
        assert O.incrementer_circuit(x, n) == (x + 1) % (1 << n)


def test_bulk_tensors_as_printed():
    tab = {}
    with open(os.path.join(GOLD, "eq9_13_shift_tensors.txt")) as f:
        for line in f:
            p = line.split("#")[0].split()
            if p:
                tab[(p[0], int(p[1]), int(p[2]))] = np.array([float(v) for v in p[3:]]).reshape(2, 2)
    n = 4
    for name, sign in (("W", +1), ("V", -1)):
        cores = O.shift_mpo_1d(n, sign, O.PERIODIC)
        bulk = cores[1]  # a bulk site: [a_in][t][s][a_out], Eq. 12 order
        for a_in in range(2):
            for a_out in range(2):
                np.testing.assert_array_equal(bulk[a_in, :, :, a_out], tab[(name, a_in, a_out)])


def _perm_matrix(n, f):
    N = 1 << n
    P = np.zeros((N, N))
    for x in range(N):
        y = f(x)
        if y is not None:
            P[y, x] = 1.0
    return P


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("bc", BCS)
def test_shift_mpo_1d_is_brute_force_shift(n, bc):
    N = 1 << n
    inc = (lambda x: (x + 1) % N) if bc == O.PERIODIC else (lambda x: x + 1 if x + 1 < N else None)
    dec = (lambda x: (x - 1) % N) if bc == O.PERIODIC else (lambda x: x - 1 if x >= 1 else None)
    Sp = O.line_operator(O.shift_mpo_1d(n, +1, bc), n)
    Sm = O.line_operator(O.shift_mpo_1d(n, -1, bc), n)
    np.testing.assert_array_equal(Sp, _perm_matrix(n, inc))
    np.testing.assert_array_equal(Sm, _perm_matrix(n, dec))
    if bc == O.PERIODIC:  # Sec. 3.1: S^- is the adjoint of S^+
        np.testing.assert_array_equal(Sm, Sp.T)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_eq11_terminal_as_printed_drops_the_overflow(n):
    """The terminal tensor of Eq. 11 keeps only carry-out 0, so the printed
    MPO maps |2^n - 1> to 0 instead of |0>: a zero-outside shift."""
    N = 1 << n
    S = O.line_operator(O.shift_mpo_1d(n, +1, O.PERIODIC, literal_eq11=True), n)
    np.testing.assert_array_equal(S, _perm_matrix(n, lambda x: x + 1 if x + 1 < N else None))
    assert np.all(S[:, N - 1] == 0.0)


def _stencil(n, bc):
    N = 1 << n
    B = np.zeros((N * N, N * N))
    for x in range(N):
        for z in range(N):
            i = x * N + z
            B[i, i] = -4.0
            for dx, dz in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, zz = x + dx, z + dz
                if bc == O.PERIODIC:
                    xx %= N
                    zz %= N
                elif not (0 <= xx < N and 0 <= zz < N):
                    continue
                B[i, xx * N + zz] += 1.0
    return B


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_laplacian_mpo_is_five_point_stencil(n, order, bc):
    L = O.laplacian_mpo(n, order, bc)
    assert all(w.shape[0] <= 5 and w.shape[3] <= 5 for w in L)
    np.testing.assert_array_equal(O.grid_operator(L, n, order), _stencil(n, bc))


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("bc", BCS)
def test_laplacian_equals_sum_of_lifted_shifts(n, order, bc):
    """Eq. 16 as a sum of the Eq. 14-15 lifts."""
    tot = -4.0 * np.eye(1 << (2 * n))
    for ax in ("x", "z"):
        for sg in (+1, -1):
            tot += O.grid_operator(O.shift_mpo_2d(n, ax, sg, bc, order), n, order)
    np.testing.assert_array_equal(O.grid_operator(O.laplacian_mpo(n, order, bc), n, order), tot)


@pytest.mark.parametrize("order", ORDERS)
def test_encoding_round_trip_and_bits(order):
    n = 3
    N = 1 << n
    rng = np.random.default_rng(0)
    u = rng.standard_normal((N, N))
    t = O.dense_to_tensor(u, n, order)
    np.testing.assert_array_equal(O.tensor_to_dense(t, n, order), u)
    for x in range(N):
        for z in range(N):
            assert t[tuple(O.site_bits(x, z, n, order))] == u[x, z]
    # x = 6 = 110b, z = 1 = 001b; sites least significant bit first (Eq. 12),
    # x register before z register (Eq. 14-15)
    if order == O.SEQUENTIAL:
        assert O.site_bits(6, 1, 3, order) == [0, 1, 1, 1, 0, 0]
    else:
        assert O.site_bits(6, 1, 3, order) == [0, 1, 1, 0, 1, 0]
