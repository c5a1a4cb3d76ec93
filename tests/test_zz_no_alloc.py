"""The allocation-free truncated SVD (qtt_svd_trunc_noalloc) against the
regular entry point (qtt_svd_trunc).

qtt_svd_trunc_noalloc serves callers that cannot allocate device memory
(their memory belongs to another allocator, or a cudaMalloc's implicit
synchronisation is not acceptable in their loop): its scratch is a static
device array inside the library, so the caller hands over only the matrix
and the output buffers.  This file is collected last so that a run stopping
at its first failure has already run every other test."""
import numpy as np
import pytest

from oracle import qtt_oracle as O

pytestmark = pytest.mark.gpu

TOL_S = 1e-12  # singular values, relative to sigma_1 (as in the parity tests)
TOL_REC = 1e-10  # reconstruction, relative to sigma_1


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2609_01904_b300 import build
    build.build()
    from paper_2609_01904_b300 import qtt
    return qtt


def _matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    A = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    return A * np.exp(-0.08 * np.arange(n))[None, :]


def _noalloc(q, A, eps, chi):
    import torch
    m, n = A.shape
    k = min(m, n)
    M = torch.as_tensor(A, device="cuda")
    U = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    S = torch.zeros((k,), dtype=torch.float64, device="cuda")
    Vt = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    r = q.qtt_svd_trunc_noalloc(M, U, S, Vt, eps, chi)
    U = U.cpu().numpy().reshape(-1)[: m * r].reshape(m, r)
    return U, S.cpu().numpy()[:r], Vt.cpu().numpy()[:r], r


def test_noalloc_svd_matches_the_regular_entry_point_on_two_calls_in_a_row(q):
    import torch
    ctx = q.qtt_ctx_create(n=8, chi_max=128)
    for m, n, seed, eps, chi in ((300, 100, 1, 1e-9, 0), (90, 400, 2, 1e-6, 40)):
        A = _matrix(m, n, seed)
        U0, S0, Vt0, r0 = q.qtt_svd_trunc(ctx, torch.as_tensor(A, device="cuda"), eps, chi)
        U0, S0, Vt0 = U0.cpu().numpy(), S0.cpu().numpy(), Vt0.cpu().numpy()
        U1, S1, Vt1, r1 = _noalloc(q, A, eps, chi)
        assert r1 == r0
        s1 = float(S0[0])
        np.testing.assert_allclose(S1, S0, rtol=0, atol=TOL_S * s1)
        rec0 = U0 @ np.diag(S0) @ Vt0
        rec1 = U1 @ np.diag(S1) @ Vt1
        assert np.linalg.norm(rec1 - rec0) <= TOL_REC * s1
        # singular vectors agree up to sign, weighted by their values
        sg = np.sign(np.sum(U0 * U1, axis=0))
        np.testing.assert_allclose(U1 * sg * S1, U0 * S0, rtol=0, atol=TOL_REC * s1)


def test_noalloc_svd_rejects_sizes_beyond_its_scratch(q):
    import torch
    M = torch.zeros((600, 20), dtype=torch.float64, device="cuda")
    U = torch.zeros((600, 20), dtype=torch.float64, device="cuda")
    S = torch.zeros((20,), dtype=torch.float64, device="cuda")
    Vt = torch.zeros((20, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QttError) as ei:
        q.qtt_svd_trunc_noalloc(M, U, S, Vt, 1e-8, 0)
    assert ei.value.status == q.QTT_EINVAL
    assert "static scratch" in str(ei.value)


@pytest.mark.parametrize("m,n,seed,eps,chi", [(128, 128, 5, 1e-9, 0), (512, 128, 6, 1e-7, 0), (128, 512, 7, 1e-7, 50),
                                             (1, 1, 8, 0.0, 0), (1, 37, 9, 0.0, 0), (64, 64, 0, 1e-8, 0)])
def test_noalloc_svd_matches_the_oracle_rule_and_numpy_singular_values(q, m, n, seed, eps, chi):
    """Against the oracle's truncation rule (Sec. 4.3) and the singular values
    numpy's LAPACK SVD returns: the square branch (no QR), both sides at the
    limit of the scratch (512 x 128 and 128 x 512), a 1 x 1 and a 1 x n
    matrix, and the zero matrix (seed 0), each called twice in a row."""
    A = _matrix(m, n, seed) if seed else np.zeros((m, n))
    s_ref = np.linalg.svd(A, compute_uv=False)
    r_ref = O.trunc_rank(s_ref, eps, chi if chi > 0 else 1 << 30)
    for _ in range(2):
        U, S, Vt, r = _noalloc(q, A, eps, chi)
        assert r == r_ref
        scale = max(float(s_ref[0]), 1e-300)
        np.testing.assert_allclose(S, s_ref[:r], rtol=0, atol=TOL_S * scale)
        best = float(np.sqrt(np.sum(s_ref[r:] ** 2)))
        err = float(np.linalg.norm(U @ np.diag(S) @ Vt - A))
        assert abs(err - best) <= TOL_REC * scale
        if s_ref[0] == 0.0:
            assert not S.any() and not (U @ np.diag(S) @ Vt).any()
