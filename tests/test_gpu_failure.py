"""Failure detection on the device, without faulting the GPU.

Every wait a kernel makes on another CTA of its launch is bounded: it gives
up after the context's wait limit, records QTT_ETIMEOUT in the device status
word and returns.  The FP64 Jacobi SVD records QTT_ENOCONV when it reaches its
sweep limit.  These tests make both run out on purpose, on small matrices,
through qtt_set_limits: a wait limit of one nanosecond (no wait between CTAs
can be met that fast) and a sweep limit of one (a random matrix needs more).
Each checks that the status comes back through the C ABI, that the context
stays usable, and that the next call, with the limits restored, gives the
oracle's answer again."""
import numpy as np
import pytest

from oracle import qtt_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2609_01904_b300 import build
    build.build()
    from paper_2609_01904_b300 import qtt
    return qtt


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _svd_ok(q, ctx, A):
    U, S, Vt, r = q.qtt_svd_trunc(ctx, _t(A), 0.0, 0)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert r == O.trunc_rank(s_ref, 0.0, 1 << 30)
    np.testing.assert_allclose(S.cpu().numpy(), s_ref[:r], rtol=0, atol=1e-12 * s_ref[0])


def test_wait_limit_runs_out_and_the_context_recovers(q):
    """The cooperative FP64 Jacobi of a 96 x 96 matrix waits on the rounds of
    other CTAs; with a 1 ns limit the first such wait gives up."""
    ctx = q.qtt_ctx_create(n=6, chi_max=64)
    A = np.random.default_rng(3).standard_normal((96, 96))
    _svd_ok(q, ctx, A)
    q.qtt_set_limits(ctx, 1e-9, 0)
    with pytest.raises(q.QttError) as e:
        q.qtt_svd_trunc(ctx, _t(A), 0.0, 0)
    assert e.value.status == q.QTT_ETIMEOUT
    q.qtt_ctx_sync(ctx)  # the status word was reset by the failing call
    q.qtt_set_limits(ctx, 0.0, 0)
    _svd_ok(q, ctx, A)
    _svd_ok(q, ctx, A)


def test_sweep_limit_runs_out_and_the_context_recovers(q):
    ctx = q.qtt_ctx_create(n=6, chi_max=64)
    A = np.random.default_rng(4).standard_normal((80, 80))
    q.qtt_set_limits(ctx, 0.0, 1)
    with pytest.raises(q.QttError) as e:
        q.qtt_svd_trunc(ctx, _t(A), 0.0, 0)
    assert e.value.status == q.QTT_ENOCONV
    q.qtt_set_limits(ctx, 0.0, 0)
    _svd_ok(q, ctx, A)


def test_step_after_a_timed_out_step_matches_the_oracle(q):
    """A whole FP64 step with a 1 ns wait limit reports QTT_ETIMEOUT (the
    cooperative QR and Jacobi kernels give up); with the default limit
    restored, a step from fresh states matches the oracle to 1e-10."""
    n, chi, eps = 4, 16, 1e-9
    N = 1 << n
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=8, eps_c=1e-8)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.1), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.1), 1e-14, chi)
    q.qtt_set_limits(ctx, 1e-9, 0)
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    with pytest.raises(q.QttError) as e:
        q.qtt_step(L, C, lam2, prev, cur, (3, 5), 0.25)
        q.qtt_ctx_sync(ctx)
    assert e.value.status == q.QTT_ETIMEOUT
    q.qtt_set_limits(ctx, 0.0, 0)
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    q.qtt_step(L, C, lam2, prev, cur, (3, 5), 0.25)
    want = O.mps_step(O.laplacian_mpo(n, "interleaved", "periodic"), O.velocity_mps(c, n, "interleaved", 1e-8, 8),
                      lam2, prev_h, cur_h, eps, chi, (3, 5), 0.25, n, "interleaved")
    import torch
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(cur, out)
    q.qtt_ctx_sync(ctx)
    ref = O.mps_to_dense(want, n, "interleaved")
    assert q.qtt_mps_ranks(cur) == O.mps_ranks(want)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_set_limits_rejects_bad_arguments(q):
    ctx = q.qtt_ctx_create(n=3, chi_max=8)
    with pytest.raises(q.QttError) as e:
        q.qtt_set_limits(ctx, 1e9, 0)
    assert e.value.status == q.QTT_EINVAL
