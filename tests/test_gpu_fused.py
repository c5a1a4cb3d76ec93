"""The fused step (Eq. 7 with A = 2I + lambda^2 C^2 L applied as one MPO,
qtt_a_operator_mpo + qtt_step_fused) against the oracle's mirror of the same
variant (oracle.a_operator_mpo, oracle.mps_step_fused), mode for mode.

Tolerances as for the two-zip-up step: FP64 form ranks equal and 1e-10
relative L2; FP32 form the bounds of tests/fp32_bounds.py.  The untruncated
fused step reproduces the dense Eq. 2 update (Table 1)."""
import math

import numpy as np
import pytest

from fp32_bounds import gaps, ranks_ok, tol32
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


def _dense(q, psi, N):
    import torch
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(psi, out)
    q.qtt_ctx_sync(psi.ctx)
    return out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_step_from_random_state_matches_the_oracle_mirror(q, order, bc, prec):
    n, chi, eps = 5, 16, 1e-6
    N = 1 << n
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=chi, eps=eps, chi_c=8, eps_c=1e-8, prec=prec)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    A = q.qtt_a_operator_mpo(L, C, lam2)
    Ao = O.a_operator_mpo(O.laplacian_mpo(n, order, bc), O.velocity_mps(c, n, order, 1e-8, 8), lam2)
    assert q.qtt_mpo_bonds(A) == [1] + [a.shape[3] for a in Ao]
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.15), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.15), 1e-14, chi)
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    src = (N // 2 + 1, 3)
    q.qtt_step_fused(A, prev, cur, src, 0.37)
    st = []
    want = O.mps_step_fused(Ao, prev_h, cur_h, eps, chi, src, 0.37, n, order, st)
    got_r, want_r = q.qtt_mps_ranks(cur), O.mps_ranks(want)
    err = _rel(_dense(q, cur, N), O.mps_to_dense(want, n, order))
    if prec == "fp64":
        assert got_r == want_r
        assert err < RTOL, err
    else:
        tol, deg = tol32(st, eps)
        print(f"fused fp32 {order} {bc}: rel_l2 {err:.3e} tol {tol:.1e} gaps {gaps(st)}")
        assert ranks_ok(got_r, want_r, st, eps), (got_r, want_r)
        assert not deg and err < tol, (err, tol)
    assert _rel(_dense(q, prev, N), O.mps_to_dense(cur_h, n, order)) < 1e-13


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_untruncated_fused_gpu_step_equals_dense_fdtd(q, order, bc):
    """Table 1 with Eq. 7's operator in one zip-up: chi = inf, eps = 0."""
    import torch
    n, N = 3, 8
    rng = np.random.default_rng(5)
    c = rng.uniform(1500.0, 3000.0, (N, N))
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=64, eps=0.0, chi_c=64, eps_c=1e-300)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    A = q.qtt_a_operator_mpo(L, C, lam2)
    c2r = _dense(q, C, N)
    prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    upo, uco = np.zeros((N, N)), np.zeros((N, N))
    for k in range(20):
        amp = math.sin(0.4 * k) + 0.05 * k
        q.qtt_step_fused(A, prev, cur, (2, 5), amp)
        upo, uco = uco, O.fdtd_step(upo, uco, c2r, lam2, bc, (2, 5), amp)
    assert _rel(_dense(q, cur, N), uco) < 1e-11


def test_fused_qtt64_teacher_forced_every_5th_step(q):
    """Every 5th step of the 64 x 64 workload's 300 in the fused form, FP64,
    each from the oracle's fused-form state."""
    wl = W.config(0)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    A = q.qtt_a_operator_mpo(L, C, lam2)
    Ao = O.a_operator_mpo(O.laplacian_mpo(n, wl.order, wl.bc), O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c),
                          lam2)
    src = (N // 2 + 1, N // 2)
    po, co = O.zero_mps(2 * n), O.zero_mps(2 * n)
    worst = 0.0
    for k in range(wl.steps):
        nxt = O.mps_step_fused(Ao, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order)
        if k % 5 == 4:
            prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
            q.qtt_step_fused(A, prev, cur, src, float(amps[k]))
            assert q.qtt_mps_ranks(cur) == O.mps_ranks(nxt), k
            worst = max(worst, _rel(_dense(q, cur, N), O.mps_to_dense(nxt, n, wl.order)))
        po, co = co, nxt
    print(f"fused qtt64 fp64: worst rel_l2 {worst:.2e}")
    assert worst < RTOL, worst
