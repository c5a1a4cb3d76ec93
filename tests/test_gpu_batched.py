"""Batched shots (one step of Eq. 17 for many independent sources, each with
its own bond cap) against the FP64 oracle, shot by shot.

Every shot starts from its own seeded right-canonical pair (u^{k-1}, u^k),
teacher-forced from the oracle at each step (the truncated dynamics is
chaotic once chi binds, so parity is per step).  FP64 shots must match the
oracle within 1e-10 relative L2 with identical ranks; FP32-form shots within
the FP32 form's bounds (tests/fp32_bounds.py: min(2e-5 + 1e-6 / h, 1e-4), h
the smallest relative gap at a discarding cut of that shot's step; ranks
within 2 plus the values near eps sigma_1)."""
import numpy as np
import pytest

from fp32_bounds import gaps, ranks_ok, tol32
from oracle import qtt_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-10


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


def _dense(q, psi, N):
    import torch
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(psi, out)
    q.qtt_ctx_sync(psi.ctx)
    return out.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)





def _state(n, chi, seed):
    return O.tt_round(W.random_tt_cores(2 * n, chi, seed, decay=0.1), 1e-14, chi)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,chis,order,bc", [
    (5, [8, 16, 12, 16, 8, 24], "interleaved", "periodic"),
    (5, [16, 4, 8], "sequential", "zero"),
    (4, [4, 8, 16, 8, 4, 8, 16, 8, 4, 12, 6], "interleaved", "periodic"),  # 11 shots on 8 pool streams
])
def test_batched_step_matches_oracle_shot_by_shot(q, prec, n, chis, order, bc):
    N = 1 << n
    eps = 1e-6
    ns = len(chis)
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    chi_top = max(chis)
    batch = q.qtt_batch_create(n, ns, chis, order=order, bc=bc, chi_max=chi_top, eps=eps, chi_c=12, eps_c=1e-8,
                               prec=prec)
    ctx0 = batch.ctxs[0]
    L = q.qtt_laplacian_mpo(ctx0)
    C = q.qtt_velocity_mps(ctx0, _t(c))
    Lo = O.laplacian_mpo(n, order, bc)
    Co = O.velocity_mps(c, n, order, 1e-8, 12)
    srcs = [((N // 128 + s * max(N // ns, 1)) % N, 2 + s % 3) for s in range(ns)]
    po = [_state(n, chis[s], 100 + 2 * s) for s in range(ns)]
    co = [_state(n, chis[s], 101 + 2 * s) for s in range(ns)]
    for k in range(3):
        prev = [q.qtt_mps_from_cores(batch.ctxs[s], po[s]) for s in range(ns)]
        cur = [q.qtt_mps_from_cores(batch.ctxs[s], co[s]) for s in range(ns)]
        amps = [0.3 + 0.1 * s - 0.2 * k for s in range(ns)]
        q.qtt_step_batched(batch, L, C, lam2, prev, cur, srcs, amps)
        for s in range(ns):
            st = []
            want = O.mps_step(Lo, Co, lam2, po[s], co[s], eps, chis[s], srcs[s], amps[s], n, order, st)
            got_r, want_r = q.qtt_mps_ranks(cur[s]), O.mps_ranks(want)
            assert max(got_r) <= chis[s]
            err = _rel(_dense(q, cur[s], N), O.mps_to_dense(want, n, order))
            if prec == "fp64":
                assert got_r == want_r, (k, s)
                assert err < RTOL, (k, s, err)
            else:
                tol, deg = tol32(st, eps)
                assert ranks_ok(got_r, want_r, st, eps), (k, s, got_r, want_r)
                assert deg or err < tol, (k, s, err, tol, gaps(st))
            # psi_prev now holds u^k
            assert _rel(_dense(q, prev[s], N), O.mps_to_dense(co[s], n, order)) < 1e-13
            po[s], co[s] = co[s], want


def test_batched_free_run_equals_the_same_shots_stepped_one_by_one(q):
    """A source-driven run of 30 steps from zero fields: each batched shot
    follows the trajectory of the same shot stepped alone with qtt_step, to
    within FP64 rounding (the two differ only in how many CTAs the
    cooperative kernels use), before the chi cap makes the dynamics chaotic."""
    n, N, eps = 5, 32, 1e-12
    chis = [32, 32, 32, 32]
    c = W.layered_model(n, 40.0, 3)
    lam2 = (0.5 / c.max()) ** 2
    batch = q.qtt_batch_create(n, len(chis), chis, chi_max=32, eps=eps, chi_c=12, eps_c=1e-8)
    ref_ctx = q.qtt_ctx_create(n=n, chi_max=32, eps=eps, chi_c=12, eps_c=1e-8)
    L = q.qtt_laplacian_mpo(batch.ctxs[0])
    C = q.qtt_velocity_mps(batch.ctxs[0], _t(c))
    Lr = q.qtt_laplacian_mpo(ref_ctx)
    Cr = q.qtt_velocity_mps(ref_ctx, _t(c))
    srcs = [(4 + 7 * s, 2 + s) for s in range(len(chis))]
    prev = [q.qtt_mps_create_zero(x) for x in batch.ctxs]
    cur = [q.qtt_mps_create_zero(x) for x in batch.ctxs]
    rp = [q.qtt_mps_create_zero(ref_ctx) for _ in chis]
    rc = [q.qtt_mps_create_zero(ref_ctx) for _ in chis]
    for k in range(30):
        amps = [np.sin(0.3 * k + s) for s in range(len(chis))]
        q.qtt_step_batched(batch, L, C, lam2, prev, cur, srcs, amps)
        for s in range(len(chis)):
            q.qtt_step(Lr, Cr, lam2, rp[s], rc[s], srcs[s], amps[s])
    for s in range(len(chis)):
        assert _rel(_dense(q, cur[s], N), _dense(q, rc[s], N)) < 1e-10


def test_batched_step_rejects_a_state_of_another_shot(q):
    batch = q.qtt_batch_create(3, 2, [4, 8], chi_max=8, eps=1e-8)
    L = q.qtt_laplacian_mpo(batch.ctxs[0])
    C = q.qtt_velocity_mps(batch.ctxs[0], _t(np.full((8, 8), 1500.0)))
    prev = [q.qtt_mps_create_zero(batch.ctxs[0]), q.qtt_mps_create_zero(batch.ctxs[0])]
    cur = [q.qtt_mps_create_zero(batch.ctxs[0]), q.qtt_mps_create_zero(batch.ctxs[1])]
    with pytest.raises(q.QttError) as e:
        q.qtt_step_batched(batch, L, C, 1e-8, prev, cur)
    assert e.value.status == q.QTT_EINVAL


def test_batched_graph_replays_equal_batched_steps(q):
    """The same batch stepped through graph replays (qtt_batch_set_graphs)
    reproduces the plainly launched batch bit for bit."""
    n, N, eps = 5, 32, 1e-9
    chis = [16, 8, 32, 16, 8]
    c = W.layered_model(n, 40.0, 3)
    lam2 = (0.5 / c.max()) ** 2
    srcs = [(3 + 5 * s, 2 + s) for s in range(len(chis))]
    out = []
    for graphs in (False, True):
        batch = q.qtt_batch_create(n, len(chis), chis, chi_max=32, eps=eps, chi_c=12, eps_c=1e-8, prec="fp32")
        q.qtt_batch_set_graphs(batch, graphs)
        L = q.qtt_laplacian_mpo(batch.ctxs[0])
        C = q.qtt_velocity_mps(batch.ctxs[0], _t(c))
        prev = [q.qtt_mps_create_zero(x) for x in batch.ctxs]
        cur = [q.qtt_mps_create_zero(x) for x in batch.ctxs]
        for k in range(12):
            q.qtt_step_batched(batch, L, C, lam2, prev, cur, srcs, [np.sin(0.5 * k + s) for s in range(len(chis))])
        out.append([_dense(q, x, N) for x in cur])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
