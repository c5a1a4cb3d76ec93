"""The 3D extension (a context with dims = 3: 3n sites, the 7-point
Laplacian) against the 3D oracle (oracle/qtt3d.py).

FP64 form: ranks equal and dense fields within 1e-10 relative L2 of the
oracle; the reduced-precision form within the bounds of tests/fp32_bounds.py.
The untruncated 3D step reproduces the dense 7-point update, on the GPU
(qtt_fdtd_step_3d) and in the oracle."""
import math

import numpy as np
import pytest

from fp32_bounds import gaps, ranks_ok, tol32
from oracle import qtt3d as O3
from oracle import qtt_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-10
INF = 1 << 30


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


def _dense3(q, psi, N):
    import torch
    out = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(psi, out)
    q.qtt_ctx_sync(psi.ctx)
    return out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_3d_laplacian_mpo_bonds_match_oracle(q, order, bc, n):
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=8, dims=3)
    L = q.qtt_laplacian_mpo(ctx)
    assert q.qtt_mpo_bonds(L) == [1] + [w.shape[3] for w in O3.laplacian_mpo(n, order, bc)]


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("n,chi,eps", [(2, 64, 0.0), (3, 16, 1e-6), (4, 32, 1e-8)])
def test_3d_tt_svd_sample_and_to_dense_match_oracle(q, order, n, chi, eps):
    import torch
    N = 1 << n
    rng = np.random.default_rng(n + 10)
    x = np.linspace(0, 1, N)
    u = (np.sin(5 * x)[:, None, None] * np.cos(3 * x)[None, :, None] * (1 + x)[None, None, :]
         + 0.2 * rng.standard_normal((N, N, N)) * np.exp(-30 * (x[:, None, None] - 0.5) ** 2))
    ctx = q.qtt_ctx_create(n=n, order=order, chi_max=chi, eps=eps, dims=3)
    psi = q.qtt_mps_from_dense(ctx, _t(u))
    ref = O3.state_from_dense(u, n, order, eps, chi)
    assert q.qtt_mps_ranks(psi) == O.mps_ranks(ref)
    want = O3.mps_to_dense(ref, n, order)
    assert _rel(_dense3(q, psi, N), want) < RTOL
    pts = rng.integers(0, N, (40, 3))
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    q.qtt_sample_3d(psi, *[torch.as_tensor(np.ascontiguousarray(pts[:, a]), device="cuda") for a in range(3)], out)
    np.testing.assert_allclose(out.cpu().numpy(), O3.mps_sample(ref, n, order, pts), rtol=0,
                               atol=RTOL * np.abs(want).max())


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_untruncated_3d_gpu_step_equals_gpu_and_oracle_dense_update(q, order, bc):
    import torch
    n, N = 2, 4
    rng = np.random.default_rng(6)
    c = rng.uniform(1500.0, 3000.0, (N, N, N))
    lam2 = (0.4 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=64, eps=0.0, chi_c=64, eps_c=1e-300, dims=3)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    c2r = _dense3(q, C, N)
    prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    up = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    c2t = _t(c2r)
    upo, uco = np.zeros((N, N, N)), np.zeros((N, N, N))
    src = (1, 2, 3)
    for k in range(20):
        amp = math.sin(0.4 * k) + 0.05 * k
        q.qtt_step(L, C, lam2, prev, cur, src, amp)
        q.qtt_fdtd_step_3d(ctx, c2t, lam2, up, uc, un, src, amp)
        up, uc, un = uc, un, up
        upo, uco = uco, O3.fdtd_step(upo, uco, c2r, lam2, bc, src, amp)
    q.qtt_ctx_sync(ctx)
    assert _rel(uc.cpu().numpy(), uco) < 1e-13
    assert _rel(_dense3(q, cur, N), uco) < 1e-11


def _random_state(n, chi, seed):
    return O.tt_round(W.random_tt_cores(3 * n, chi, seed, decay=0.15), 1e-14, chi)


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_3d_step_from_random_state_matches_oracle(q, order, bc, prec):
    n, chi, eps = 3, 16, 1e-6
    N = 1 << n
    c = W.layered_model_3d(n, 100.0, 3)
    lam2 = (0.4 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=chi, eps=eps, chi_c=8, eps_c=1e-8, prec=prec, dims=3)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev_h, cur_h = _random_state(n, chi, 1), _random_state(n, chi, 2)
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    src = (N // 2 + 1, 2, 3)
    q.qtt_step(L, C, lam2, prev, cur, src, 0.37)
    st = []
    want = O3.mps_step(O3.laplacian_mpo(n, order, bc), O3.velocity_mps(c, n, order, 1e-8, 8), lam2, prev_h, cur_h,
                       eps, chi, src, 0.37, n, order, st)
    got_r, want_r = q.qtt_mps_ranks(cur), O.mps_ranks(want)
    err = _rel(_dense3(q, cur, N), O3.mps_to_dense(want, n, order))
    if prec == "fp64":
        assert got_r == want_r
        assert err < RTOL, err
    else:
        tol, deg = tol32(st, eps)
        print(f"3d fp32 {order} {bc}: rel_l2 {err:.3e} tol {tol:.1e} gaps {gaps(st)}")
        assert ranks_ok(got_r, want_r, st, eps), (got_r, want_r)
        assert not deg and err < tol, (err, tol)


def test_3d_workload_teacher_forced_steps_match_oracle(q):
    """The 3D workload at 16^3 (n = 4, chi = 64, eps = 1e-6, Ricker source):
    every 10th of its first 100 steps, FP64, from the oracle's state."""
    wl = W.qtt3d_run(4)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c, 100)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, dims=3)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    Lo = O3.laplacian_mpo(n, wl.order, wl.bc)
    Co = O3.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    assert q.qtt_mps_ranks(C) == O.mps_ranks(Co)
    src = wl.sources[0]
    po, co = O.zero_mps(3 * n), O.zero_mps(3 * n)
    worst = 0.0
    for k in range(100):
        nxt = O3.mps_step(Lo, Co, lam2, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order)
        if k % 10 == 9:
            prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
            q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
            assert q.qtt_mps_ranks(cur) == O.mps_ranks(nxt), k
            worst = max(worst, _rel(_dense3(q, cur, N), O3.mps_to_dense(nxt, n, wl.order)))
        po, co = co, nxt
    print(f"3d workload n=4: worst rel_l2 {worst:.2e}, final max rank {max(O.mps_ranks(co))}")
    assert worst < RTOL, worst


def test_3d_context_rejects_2d_point_calls(q):
    import torch
    ctx = q.qtt_ctx_create(n=2, chi_max=8, dims=3)
    psi = q.qtt_mps_create_zero(ctx)
    with pytest.raises(q.QttError) as e:
        q.qtt_inject_source(psi, 1, 1, 1.0)
    assert e.value.status == q.QTT_EINVAL
    with pytest.raises(q.QttError) as e:
        q.qtt_inject_source_3d(psi, 1, 4, 1, 1.0)
    assert e.value.status == q.QTT_EINVAL
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(q.QttError):
        q.qtt_sample(psi, z, z, torch.zeros(1, dtype=torch.float64, device="cuda"))
