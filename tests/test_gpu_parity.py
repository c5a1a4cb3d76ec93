"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: the FP64 form must match the oracle within 1e-10 relative L2 on
dense fields and samples.  Cores are never compared (they are defined up to
gauge and sign); ranks are compared exactly, singular values to 1e-12 of
sigma_1.  Inputs are seeded and shared; expected values come from oracle/."""
import math

import numpy as np
import pytest

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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("m,n,rank", [(7, 5, 5), (5, 9, 5), (64, 40, 40), (40, 200, 40), (300, 130, 130),
                                      (130, 640, 130), (96, 96, 12), (257, 33, 33)])
def test_svd_trunc_matches_oracle_rule_and_reconstructs(q, m, n, rank):
    ctx = q.qtt_ctx_create(n=8, chi_max=128)
    rng = np.random.default_rng(m * 1000 + n)
    A = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    A *= np.exp(-0.25 * np.arange(n))[None, :]
    s_ref = np.linalg.svd(A, compute_uv=False)
    for eps, chi in ((0.0, 0), (1e-6, 0), (1e-3, 7)):
        U, S, Vt, r = q.qtt_svd_trunc(ctx, _t(A), eps, chi)
        U, S, Vt = U.cpu().numpy(), S.cpu().numpy(), Vt.cpu().numpy()
        r_ref = O.trunc_rank(s_ref, eps, chi if chi > 0 else INF)
        assert r == r_ref
        np.testing.assert_allclose(S, s_ref[:r], rtol=0, atol=1e-12 * s_ref[0])
        # the factor built from the Jacobi rotations is orthogonal to rounding;
        # the other one is (rotated matrix) / sigma, accurate where weighted by sigma
        J, D = (U.T, Vt) if m <= n else (Vt, U.T)
        np.testing.assert_allclose(J @ J.T, np.eye(r), atol=1e-12)
        SD = S[:, None] * D
        np.testing.assert_allclose(SD @ SD.T, np.diag(S ** 2), atol=1e-12 * s_ref[0] ** 2)
        best = np.sqrt(np.sum(s_ref[r:] ** 2))
        err = np.linalg.norm(U @ np.diag(S) @ Vt - A)
        assert abs(err - best) <= 1e-10 * s_ref[0]


def test_svd_trunc_zero_and_rank_one(q):
    ctx = q.qtt_ctx_create(n=4, chi_max=16)
    U, S, Vt, r = q.qtt_svd_trunc(ctx, _t(np.zeros((6, 4))), 1e-8, 0)
    assert r == 1 and float(S[0]) == 0.0
    v = np.arange(1.0, 7.0)
    U, S, Vt, r = q.qtt_svd_trunc(ctx, _t(np.outer(v, [1.0, -2.0, 0.5])), 1e-12, 0)
    assert r == 1
    assert abs(float(S[0]) - np.linalg.norm(v) * math.sqrt(1 + 4 + 0.25)) < 1e-12 * float(S[0])


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
@pytest.mark.parametrize("n", [2, 4, 6])
def test_laplacian_mpo_bonds_match_oracle(q, order, bc, n):
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=8)
    L = q.qtt_laplacian_mpo(ctx)
    ref = [1] + [w.shape[3] for w in O.laplacian_mpo(n, order, bc)]
    assert q.qtt_mpo_bonds(L) == ref


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("n,chi,eps", [(3, 64, 0.0), (5, 8, 1e-8), (6, 16, 1e-4), (8, 32, 1e-6)])
def test_tt_svd_sample_and_to_dense_match_oracle(q, order, n, chi, eps):
    import torch
    N = 1 << n
    rng = np.random.default_rng(n)
    x = np.linspace(0, 1, N)
    u = np.sin(7 * x)[:, None] * np.cos(3 * x)[None, :] + 0.3 * rng.standard_normal((N, N)) * np.exp(
        -40 * (x[:, None] - 0.5) ** 2 - 30 * (x[None, :] - 0.4) ** 2)
    ctx = q.qtt_ctx_create(n=n, order=order, chi_max=chi, eps=eps)
    psi = q.qtt_mps_from_dense(ctx, _t(u))
    ref = O.state_from_dense(u, n, order, eps, chi)
    assert q.qtt_mps_ranks(psi) == O.mps_ranks(ref)
    got = _dense(q, psi, N)
    want = O.mps_to_dense(ref, n, order)
    assert _rel(got, want) < RTOL
    ix = rng.integers(0, N, 50)
    iz = rng.integers(0, N, 50)
    out = torch.zeros(50, dtype=torch.float64, device="cuda")
    q.qtt_sample(psi, torch.as_tensor(ix, device="cuda"), torch.as_tensor(iz, device="cuda"), out)
    np.testing.assert_allclose(out.cpu().numpy(), O.mps_sample(ref, n, order, ix, iz), rtol=0,
                               atol=RTOL * np.abs(want).max())
    # host-buffer entry: same result
    psi2 = q.qtt_mps_from_dense(ctx, u)
    assert _rel(_dense(q, psi2, N), want) < RTOL


@pytest.mark.parametrize("cfg", [1, 2])
def test_velocity_mps_matches_oracle(q, cfg):
    wl = W.config(cfg)
    n = 6 if cfg == 1 else 7
    c = W.layered_model(n, wl.dh, wl.seed)
    ctx = q.qtt_ctx_create(n=n, order=wl.order, chi_max=32, chi_c=24, eps_c=1e-8)
    c2 = q.qtt_velocity_mps(ctx, _t(c))
    ref = O.velocity_mps(c, n, wl.order, 1e-8, 24)
    assert q.qtt_mps_ranks(c2) == O.mps_ranks(ref)
    assert _rel(_dense(q, c2, 1 << n), O.mps_to_dense(ref, n, wl.order)) < RTOL


def _random_right_canonical(n, chi, seed, order):
    """Seeded random state brought to the form the stepper keeps (oracle round)."""
    d = 2 * n
    cores = W.random_tt_cores(d, chi, seed, decay=0.15)
    return O.tt_round(cores, 1e-14, chi)


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_one_step_from_random_state_matches_oracle(q, order, bc):
    n, chi, eps = 5, 16, 1e-7
    N = 1 << n
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8)
    prev_h = _random_right_canonical(n, chi, 1, order)
    cur_h = _random_right_canonical(n, chi, 2, order)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev = q.qtt_mps_from_cores(ctx, prev_h)
    cur = q.qtt_mps_from_cores(ctx, cur_h)
    src = (N // 2 + 1, 3)
    q.qtt_step(L, C, lam2, prev, cur, src, 0.37)
    Lo = O.laplacian_mpo(n, order, bc)
    Co = O.velocity_mps(c, n, order, 1e-8, 12)
    want = O.mps_step(Lo, Co, lam2, prev_h, cur_h, eps, chi, src, 0.37, n, order)
    assert q.qtt_mps_ranks(cur) == O.mps_ranks(want)
    assert _rel(_dense(q, cur, N), O.mps_to_dense(want, n, order)) < RTOL
    assert _rel(_dense(q, prev, N), O.mps_to_dense(cur_h, n, order)) < 1e-13


@pytest.mark.parametrize("order", ["sequential", "interleaved"])
@pytest.mark.parametrize("bc", ["periodic", "zero"])
def test_untruncated_gpu_step_equals_gpu_and_oracle_fdtd(q, order, bc):
    """Table 1 on the GPU: chi = inf, eps = 0 reproduces Eq. 2."""
    import torch
    n = 3
    N = 8
    rng = np.random.default_rng(5)
    c = rng.uniform(1500.0, 3000.0, (N, N))
    lam2 = (0.5 / c.max()) ** 2
    ctx = q.qtt_ctx_create(n=n, order=order, bc=bc, chi_max=64, eps=0.0, chi_c=64, eps_c=1e-300)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    c2r = _dense(q, C, N)
    prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc = up.clone()
    un = up.clone()
    c2t = _t(c2r)
    upo, uco = np.zeros((N, N)), np.zeros((N, N))
    for k in range(20):
        amp = math.sin(0.4 * k) + 0.05 * k
        q.qtt_step(L, C, lam2, prev, cur, (2, 5), amp)
        q.qtt_fdtd_step(ctx, c2t, lam2, up, uc, un, (2, 5), amp)
        up, uc, un = uc, un, up
        upo, uco = uco, O.fdtd_step(upo, uco, c2r, lam2, bc, (2, 5), amp)
    q.qtt_ctx_sync(ctx)
    assert _rel(uc.cpu().numpy(), uco) < 1e-13
    assert _rel(_dense(q, cur, N), uco) < 1e-11


def test_inject_source_matches_oracle(q):
    n, chi = 4, 8
    order = "interleaved"
    ctx = q.qtt_ctx_create(n=n, order=order, chi_max=chi, eps=1e-9)
    cores = _random_right_canonical(n, chi, 3, order)
    psi = q.qtt_mps_from_cores(ctx, cores)
    q.qtt_inject_source(psi, 5, 9, 2.5)
    want = O.tt_round(O.mps_sum([(1.0, cores), (2.5, O.product_state(5, 9, n, order))]), 1e-9, chi)
    assert q.qtt_mps_ranks(psi) == O.mps_ranks(want)
    assert _rel(_dense(q, psi, 1 << n), O.mps_to_dense(want, n, order)) < RTOL


def _qtt64_setup(q):
    wl = W.config(0)
    n, N = wl.n, wl.N
    c = wl.velocity()
    ctx = q.qtt_ctx_create(n=n, order=wl.order, bc=wl.bc, chi_max=wl.chi, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    # source one cell off centre, so no truncation cut falls on a degenerate pair
    src = (N // 2 + 1, N // 2)
    return wl, c, ctx, L, C, Lo, Co, src


def test_qtt64_const_every_step_of_the_run_matches_oracle(q):
    """All 300 steps of the 64x64 constant-velocity workload, teacher-forced:
    at every step the GPU starts from the oracle's state (u^{k-1}, u^k) and
    its u^{k+1} and receiver samples must match the oracle's.  (Free-running
    trajectories of the truncated scheme separate by O(1) within ~100 steps
    once the chi cap binds, whatever the implementation: a 1e-15 change of
    the input does the same to the oracle itself.)"""
    import torch
    wl, c, ctx, L, C, Lo, Co, src = _qtt64_setup(q)
    n, N = wl.n, wl.N
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c)
    rx = torch.as_tensor(np.array([r[0] for r in wl.receivers]), device="cuda")
    rz = torch.as_tensor(np.array([r[1] for r in wl.receivers]), device="cuda")
    got = torch.zeros(len(wl.receivers), dtype=torch.float64, device="cuda")
    po, co = O.zero_mps(2 * n), O.zero_mps(2 * n)
    worst, worst_tr, saturated = 0.0, 0.0, 0
    for k in range(wl.steps):
        prev, cur = q.qtt_mps_from_cores(ctx, po), q.qtt_mps_from_cores(ctx, co)
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        po, co = co, O.mps_step(Lo, Co, lam2, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order)
        assert q.qtt_mps_ranks(cur) == O.mps_ranks(co), k
        want = O.mps_to_dense(co, n, wl.order)
        worst = max(worst, _rel(_dense(q, cur, N), want))
        q.qtt_sample(cur, rx, rz, got)
        tr = O.mps_sample(co, n, wl.order, rx.cpu().numpy(), rz.cpu().numpy())
        worst_tr = max(worst_tr, np.abs(got.cpu().numpy() - tr).max() / max(np.abs(want).max(), 1e-300))
        saturated += max(O.mps_ranks(co)) == wl.chi
    assert saturated > 200  # the chi cap binds for most of the run
    assert worst < RTOL, worst
    assert worst_tr < RTOL, worst_tr


def test_qtt64_const_free_run_before_saturation_matches_oracle(q):
    """The same workload free-running for its first 40 steps (before the chi
    cap binds) stays within the FP64 tolerance of the oracle's trajectory."""
    wl, c, ctx, L, C, Lo, Co, src = _qtt64_setup(q)
    n, N = wl.n, wl.N
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c)
    prev, cur = q.qtt_mps_create_zero(ctx), q.qtt_mps_create_zero(ctx)
    po, co = O.zero_mps(2 * n), O.zero_mps(2 * n)
    for k in range(40):
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        po, co = co, O.mps_step(Lo, Co, lam2, po, co, wl.eps, wl.chi, src, float(amps[k]), n, wl.order)
    assert q.qtt_mps_ranks(cur) == O.mps_ranks(co)
    assert _rel(_dense(q, cur, N), O.mps_to_dense(co, n, wl.order)) < RTOL


def test_mps_save_load_round_trip(q, tmp_path):
    n, chi = 5, 16
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-9)
    cores = _random_right_canonical(n, chi, 7, "interleaved")
    psi = q.qtt_mps_from_cores(ctx, cores)
    path = str(tmp_path / "state.qtt")
    q.qtt_mps_save(psi, path)
    ctx2 = q.qtt_ctx_create(n=n, chi_max=chi, eps=1e-9)
    back = q.qtt_mps_load(ctx2, path)
    assert q.qtt_mps_ranks(back) == O.mps_ranks(cores)
    for a, b in zip(q.qtt_mps_get_cores(back), cores):
        assert np.array_equal(a, b)
    other = q.qtt_ctx_create(n=n + 1, chi_max=chi, eps=1e-9)
    with pytest.raises(q.QttError) as e:
        q.qtt_mps_load(other, path)
    assert e.value.status == q.QTT_EINVAL
