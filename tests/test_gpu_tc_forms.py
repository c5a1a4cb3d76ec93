"""The tensor-core forms of the step (QTT_TF32X3, QTT_TF32, QTT_BF16: the
core contractions on tcgen05, everything else as in the FP32 form) against
the FP64 oracle.

Stated tolerances, relative L2 of one step from a shared state:
* TF32X3: the FP32 form's bounds (tests/fp32_bounds.py), min(2e-5 + 1e-6 / h,
  1e-4), h the smallest relative gap at a discarding cut, steps with
  h < 1e-4 reported as degenerate at FP32 resolution (its products carry
  ~2^-21 relative error, the FP32 contractions 2^-24 plus accumulation);
* TF32 and BF16: 20 u, u the operand unit roundoff (TF32 2^-11, BF16 2^-8):
  every contraction on the path of the state (about 2 d of them: the zip-up
  carries and the round's absorptions) rounds its operands once, and the
  errors of independent sites add in quadrature, sqrt(2 d) ~ 6, with margin.
Ranks: within 2 for TF32X3; for TF32 and BF16 the rank decision at eps
itself moves with the operands' rounding (values within u sigma_1 of
eps sigma_1 may flip), so only the cap and the ordering of the field are
checked through the error bound."""
import numpy as np
import pytest

from fp32_bounds import gaps, ranks_ok, tol32
from oracle import qtt_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def _tol(prec, stats, eps):
    """(tolerance, degenerate at FP32 resolution)"""
    if prec == "tf32x3":
        return tol32(stats, eps)
    return 20 * U[prec], False


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


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("n,chi,order,bc", [(5, 16, "interleaved", "periodic"), (5, 16, "sequential", "zero"),
                                            (8, 128, "interleaved", "periodic")])
def test_tensor_core_form_one_step_from_random_state(q, prec, n, chi, order, bc):
    N = 1 << n
    eps = 1e-6
    c = W.layered_model(n, 40.0 if n < 8 else 12.5, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec=prec)
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.05), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.05), 1e-14, chi)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev = q.qtt_mps_from_cores(ctx, prev_h)
    cur = q.qtt_mps_from_cores(ctx, cur_h)
    src = (N // 2 + 1, 3)
    q.qtt_step(L, C, lam2, prev, cur, src, 0.37)
    st = []
    want = O.mps_step(O.laplacian_mpo(n, order, bc), O.velocity_mps(c, n, order, 1e-8, 12), lam2, prev_h, cur_h,
                      eps, chi, src, 0.37, n, order, st)
    got_r, want_r = q.qtt_mps_ranks(cur), O.mps_ranks(want)
    err = _rel(_dense(q, cur, N), O.mps_to_dense(want, n, order))
    tol, deg = _tol(prec, st, eps)
    print(f"{prec} n={n} chi={chi} {order} {bc}: rel_l2 {err:.3e} tol {tol:.1e} gaps {gaps(st)} "
          f"max|dr| {max(abs(a - b) for a, b in zip(got_r, want_r))}")
    assert max(got_r) <= chi
    if prec == "tf32x3":
        assert ranks_ok(got_r, want_r, st, eps), (got_r, want_r)
    assert not deg and err < tol, (err, tol, gaps(st))


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
def test_tensor_core_form_teacher_forced_on_the_qtt64_run(q, prec):
    """Every 5th step of the 64 x 64 workload's 300, each from the oracle's
    state, in the tensor-core form."""
    wl = W.config(0)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec=prec)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    src = (N // 2 + 1, N // 2)
    po, co = O.zero_mps(2 * n), O.zero_mps(2 * n)
    worst, errs, ndeg = 0.0, [], 0
    for k in range(wl.steps):
        st = []
        nxt = O.mps_step(Lo, Co, lam2, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order, st)
        if k % 5 == 4:
            prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
            q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
            e = _rel(_dense(q, cur, N), O.mps_to_dense(nxt, n, wl.order))
            errs.append(e)
            tol, deg = _tol(prec, st, wl.eps)
            ndeg += deg
            if not deg:
                worst = max(worst, e / tol)
        po, co = co, nxt
    print(f"qtt64 {prec}: worst err/tol {worst:.3f}, {ndeg} of {len(errs)} checked steps degenerate at FP32 "
          f"resolution, median err {np.median(errs):.2e}, max err {max(errs):.2e}")
    assert worst < 1.0, worst
    assert ndeg <= 0.15 * len(errs), ndeg
