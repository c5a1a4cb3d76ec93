"""Symmetry of the wavefield (both oracles): with constant c, a periodic grid
and the source at the centre (N/2, N/2), the Eq. 2 update commutes with the
exchange of x and z and with the reflection x -> N - x, so the field stays
invariant under both.  The untruncated MPS step (Table 1) keeps that to
rounding; a truncated step, whose site order breaks the x <-> z symmetry of
the cuts, keeps it to the truncation level, at most steps x eps here."""
import math

import numpy as np
import pytest

from oracle import cxx as X
from oracle import qtt_oracle as O

INF = 1 << 30
N_BITS, N, STEPS = 4, 16, 40


def _run(impl, order, eps):
    c = np.ones((N, N))
    lam2 = 0.25
    src = (N // 2, N // 2)
    if impl == "numpy":
        C = O.velocity_mps(c, N_BITS, order, 0.0, INF)
        L = O.laplacian_mpo(N_BITS, order, "periodic")
        prev = cur = O.zero_mps(2 * N_BITS)
        step = lambda p, q, a: O.mps_step(L, C, lam2, p, q, eps, INF, src, a, N_BITS, order)  # noqa: E731
        dense = lambda a: O.mps_to_dense(a, N_BITS, order)  # noqa: E731
    else:
        C = X.velocity_mps(c, N_BITS, order, 0.0, INF)
        prev = cur = X.mps_from_dense(np.zeros((N, N)), N_BITS, order, 0.0, INF)
        step = lambda p, q, a: X.mps_step(N_BITS, order, "periodic", C, lam2, p, q, eps, INF, src, a)  # noqa: E731
        dense = lambda a: X.mps_to_dense(a, N_BITS, order)  # noqa: E731
    for k in range(STEPS):
        prev, cur = cur, step(prev, cur, math.exp(-((k - 10) / 4.0) ** 2))
    return dense(cur)


@pytest.mark.parametrize("impl", ["numpy", "cxx"])
@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("eps", [0.0, 1e-8])
def test_centre_source_field_is_symmetric(impl, order, eps):
    u = _run(impl, order, eps)
    nu = np.linalg.norm(u)
    tol = 1e-12 if eps == 0.0 else STEPS * eps
    assert np.linalg.norm(u - u.T) <= tol * nu
    assert np.linalg.norm(u - u[(N - np.arange(N)) % N, :]) <= tol * nu
    assert np.linalg.norm(u - u[:, (N - np.arange(N)) % N]) <= tol * nu
