"""The step replayed from a CUDA graph (qtt_step_graph) against qtt_step.

Both run the same kernels in the same order on the same inputs, so a run of
graph replays must reproduce the plain run bit for bit, in the FP64 and the
FP32 form, with a source sample that changes every step (read by the graph
from device memory) and the two state buffers exchanging roles every step."""
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


def _dense(q, psi, N):
    import torch
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(psi, out)
    q.qtt_ctx_sync(psi.ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replays_equal_plain_steps(q, prec):
    import torch
    n, chi, eps = 6, 24, 1e-7
    N = 1 << n
    c = W.layered_model(n, 20.0, 5)
    lam2 = (0.5 / c.max()) ** 2
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.2), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.2), 1e-14, chi)
    runs = []
    for graphed in (False, True):
        ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec=prec)
        L = q.qtt_laplacian_mpo(ctx)
        C = q.qtt_velocity_mps(ctx, torch.as_tensor(c, device="cuda"))
        prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
        step = q.qtt_step_graph if graphed else q.qtt_step
        for k in range(9):
            step(L, C, lam2, prev, cur, (N // 2 + 1, 3), 0.3 * np.sin(0.7 * k) + 0.05)
        runs.append((_dense(q, cur, N), _dense(q, prev, N), q.qtt_mps_ranks(cur)))
    assert runs[0][2] == runs[1][2]
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_graph_step_recaptures_for_new_arguments_and_rejects_learned_contexts(q):
    import torch
    n, chi = 4, 8
    N = 1 << n
    c = np.full((N, N), 1500.0)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-9)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, torch.as_tensor(c, device="cuda"))
    ref = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-9)
    Lr, Cr = q.qtt_laplacian_mpo(ref), q.qtt_velocity_mps(ref, torch.as_tensor(c, device="cuda"))
    a, b = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    ra, rb = q.qtt_mps_create_zero(ref), q.qtt_mps_create_zero(ref)
    for k, srcpos in enumerate([(3, 4)] * 3 + [(5, 6)] * 3):  # the source moves: a new capture
        q.qtt_step_graph(L, C, lam2, a, b, srcpos, 1.0 + k)
        q.qtt_step(Lr, Cr, lam2, ra, rb, srcpos, 1.0 + k)
    assert np.array_equal(_dense(q, b, N), _dense(q, rb, N))
    lctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-9, learned=True)
    Ll, Cl = q.qtt_laplacian_mpo(lctx), q.qtt_velocity_mps(lctx, torch.as_tensor(c, device="cuda"))
    x, y = q.qtt_mps_create_zero(lctx), q.qtt_mps_create_zero(lctx)
    with pytest.raises(q.QttError) as e:
        q.qtt_step_graph(Ll, Cl, lam2, x, y, (3, 4), 1.0)
    assert e.value.status == q.QTT_EINVAL
