"""The reduced-precision form (QTT_FP32: FP32 contractions and QR updates,
truncation SVDs as FP32 Jacobi refined to FP64 accuracy) against the FP64
oracle.

Stated tolerance (tests/fp32_bounds.py): one step from a shared state within
min(2e-5 + 1e-6 / h, 1e-4) relative L2 of the oracle, h the smallest
relative gap (sigma_r - sigma_{r+1}) / sigma_r at any truncation cut of that
step that discards a value (FP32 rounding of the contractions, ~1e-7 per
product accumulated over the step's ~60 dependent factorisations, turns a
truncated subspace by rounding / gap, weighted by the values at the cut);
a step with h < 1e-4 has a cut FP32 cannot resolve: it is counted and
reported, not held to the bound; below eps = 1e-6 (the 64 x 64 run's
eps = 1e-10) the cuts are under FP32 resolution and a step is held to the
workloads' 1e-3.  Ranks within 2 plus the number of values
within a factor 8 of eps sigma_1 (a kept / discarded decision may flip
there)."""
import numpy as np
import pytest

from fp32_bounds import gaps, ranks_ok, tol32
from oracle import qtt_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
TOL_STEP = 2e-5


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


@pytest.mark.parametrize("n,chi,order,bc", [(5, 16, "interleaved", "periodic"), (5, 16, "sequential", "zero"),
                                            (8, 128, "interleaved", "periodic")])
def test_fp32_form_one_step_from_random_state(q, n, chi, order, bc):
    N = 1 << n
    eps = 1e-6  # the FP32 form resolves cuts down to 1e-6 sigma_1
    c = W.layered_model(n, 40.0, 11) if n < 8 else W.constant_model(n, 2000.0)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec="fp32")
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
    tol, deg = tol32(st, eps)
    print(f"n={n} chi={chi} {order} {bc}: rel_l2 {err:.3e} tol {tol:.1e} gaps {gaps(st)}")
    assert ranks_ok(got_r, want_r, st, eps), (got_r, want_r)
    assert not deg and err < tol, (err, tol, gaps(st))


def test_fp32_form_every_step_of_qtt64_run(q):
    """All 300 steps of the 64x64 constant-velocity workload, teacher-forced
    from the oracle's states, in the reduced-precision form."""
    wl = W.config(0)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec="fp32")
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    src = (N // 2 + 1, N // 2)
    po, co = O.zero_mps(2 * n), O.zero_mps(2 * n)
    worst, errs, degenerate, rows = 0.0, [], [], []
    for k in range(wl.steps):
        prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        st = []
        po, co = co, O.mps_step(Lo, Co, lam2, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order, st)
        e = _rel(_dense(q, cur, N), O.mps_to_dense(co, n, wl.order))
        errs.append(e)
        tol, deg = tol32(st, wl.eps)
        rows.append((e, k, tol, deg) + gaps(st))
        if deg:
            degenerate.append(k)
        else:
            worst = max(worst, e / tol)
    for e, k, tol, deg, g, h in sorted(rows, reverse=True)[:8]:
        print(f"qtt64 fp32 step {k}: rel_l2 {e:.2e} tol {tol:.1e} degenerate {deg} gap/sigma_1 {g:.2e} "
              f"gap/sigma_r {h:.2e}")
    print(f"qtt64 fp32: worst err/tol {worst:.3f} over {wl.steps - len(degenerate)} resolvable steps, "
          f"{len(degenerate)} degenerate at FP32 resolution, median err {np.median(errs):.2e}")
    assert worst < 1.0, worst
    assert len(degenerate) <= 0.15 * wl.steps, degenerate
    assert np.median(errs) < TOL_STEP, np.median(errs)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chi256_step_on_the_512_grid(q, prec):
    """The widest bond cap of the multi-shot workload (n = 9, chi = 256, cap
    binding at the middle bonds): Jacobi SVDs of up to 512 vectors."""
    n, chi, eps = 9, 256, 1e-7
    N = 1 << n
    c = W.layered_model(n, 6.25, 4)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec=prec)
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.01), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.01), 1e-14, chi)
    assert max(O.mps_ranks(cur_h)) == chi
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev = q.qtt_mps_from_cores(ctx, prev_h)
    cur = q.qtt_mps_from_cores(ctx, cur_h)
    src = (N // 2 + 1, 3)
    q.qtt_step(L, C, lam2, prev, cur, src, 0.37)
    st = []
    want = O.mps_step(O.laplacian_mpo(n, "interleaved", "periodic"), O.velocity_mps(c, n, "interleaved", 1e-8, 12),
                      lam2, prev_h, cur_h, eps, chi, src, 0.37, n, "interleaved", st)
    got_r, want_r = q.qtt_mps_ranks(cur), O.mps_ranks(want)
    err = _rel(_dense(q, cur, N), O.mps_to_dense(want, n, "interleaved"))
    if prec == "fp64":
        assert got_r == want_r
        assert err < 1e-10, err
    else:
        tol, deg = tol32(st, eps)
        print(f"chi256 {prec}: rel_l2 {err:.3e} tol {tol:.1e} gaps {gaps(st)}")
        assert ranks_ok(got_r, want_r, st, eps), (got_r, want_r)
        assert not deg and err < tol, (err, tol, gaps(st))


def test_fp32_form_steps_from_a_mid_run_state_of_the_64_shot_workload(q):
    """Shot 1 of the 64-shot workload (n = 9, chi = 256, layered section):
    the oracle's own dense Eq. 2 run to step 1000 compressed by the oracle,
    then five FP32-form steps teacher-forced against the oracle.  The steep
    spectrum of such states has a wide cluster of near-equal tiny singular
    values, where an undamped first-order refinement diverges.  The chi cap
    falls on near-degenerate values here (relative gaps ~1e-8), where the
    truncated subspace is not unique and the gap-based tolerance is void, so
    each step is held to the workload's accuracy target, 1e-3 relative L2."""
    wl = W.config(3)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    chi = int(W.chi_per_shot(wl.seed, len(wl.sources))[1])
    assert chi == 256
    src = wl.sources[1]
    mid = 1000
    amps = wl.source_amplitudes(c, mid + 8)
    up, uc = np.zeros((N, N)), np.zeros((N, N))
    for k in range(mid):
        up, uc = uc, O.fdtd_step(up, uc, c * c, lam2, wl.bc, src, float(amps[k]))
    po = O.state_from_dense(up, n, wl.order, wl.eps, chi)
    co = O.state_from_dense(uc, n, wl.order, wl.eps, chi)
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=chi, eps=wl.eps, chi_c=wl.chi_c, eps_c=wl.eps_c,
                           prec="fp32")
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    for k in range(mid, mid + 5):
        prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        st = []
        want = O.mps_step(Lo, Co, lam2, po, co, wl.eps, chi, src, float(amps[k]), n, wl.order, st)
        got_r, want_r = q.qtt_mps_ranks(cur), O.mps_ranks(want)
        # eps = 1e-7 sits at FP32 resolution: every value within ~1e-7 sigma_1
        # of the threshold may fall either side, so ranks agree more loosely
        assert max(got_r) <= chi
        assert ranks_ok(got_r, want_r, st, wl.eps), (k, got_r, want_r)
        err = _rel(_dense(q, cur, N), O.mps_to_dense(want, n, wl.order))
        g, h = gaps(st)
        tol = min(TOL_STEP + 1e-6 / h, 1e-3)
        print(f"qtt512 shot 1 fp32 step {k}: rel_l2 {err:.3e} tol {tol:.1e} gap/sigma_1 {g:.2e} gap/sigma_r {h:.2e}")
        assert err < tol, (k, err, tol)
        po, co = co, want


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_from_the_zero_state_is_the_source_alone(q, prec):
    """Both states zero: every truncation SVD of the step factors a zero or a
    rank-one matrix (zero pivots, zero vectors), and the step leaves the
    source term alone (Eq. 17 with psi = 0)."""
    n, chi, eps = 5, 16, 1e-7
    N = 1 << n
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec=prec)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    src, amp = (N // 2 + 1, 3), 0.37
    q.qtt_step(L, C, lam2, prev, cur, src, amp)
    got = _dense(q, cur, N)
    want = np.zeros((N, N))
    want[src] = amp
    # FP32 form: the amplitude passes the FP32 QR sweep of the round
    assert np.abs(got - want).max() <= (1e-12 if prec == "fp64" else 1e-6) * amp
    assert q.qtt_mps_ranks(cur) == [1] * (2 * n + 1)
    # and with no source at all the state stays exactly zero
    z = q.qtt_mps_create_zero(ctx)
    q.qtt_step(L, C, lam2, prev, z, src, 0.0)
    assert not _dense(q, z, N).any()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_non_finite_state_is_reported(q, prec):
    """A NaN in the state reaches a singular-value spectrum and the context
    reports QTT_ENONFINITE at the next synchronisation (no silent result)."""
    n, chi = 5, 16
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-7, chi_c=12, eps_c=1e-8, prec=prec)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.05), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.05), 1e-14, chi)
    cur_h[n][0, 1, 0] = np.nan
    prev = q.qtt_mps_from_cores(ctx, prev_h)
    cur = q.qtt_mps_from_cores(ctx, cur_h)
    with pytest.raises(q.QttError) as e:
        q.qtt_step(L, C, lam2, prev, cur, (3, 3), 0.37)
        q.qtt_ctx_sync(ctx)
    assert e.value.status == q.QTT_ENONFINITE
