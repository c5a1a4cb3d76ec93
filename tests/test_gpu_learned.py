"""The learned form on the GPU against the oracle (oracle/learned.py).

Tolerances: the network runs in FP32 and the oracle in FP64 from the same
FP32 parameters, so outputs agree to ~1e-6 relative and gradients to ~1e-5
(FP32 accumulation over the batch); features to FP32 rounding.  A learned
round with given proposals is an FP64 computation and matches the oracle's
learned round to 1e-10 relative L2 with the same accept / reject decisions."""
import numpy as np
import pytest

from oracle import learned as Ln
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


def _f32(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


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


def test_param_count_matches_the_oracle_layout(q):
    assert q.qtt_mlp_param_count() == Ln.N_PARAMS


def test_mlp_forward_matches_oracle(q):
    import torch
    p = W.mlp_params(7)
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (300, Ln.N_FEAT)).astype(np.float32)
    m = q.qtt_mlp_create(p, 512)
    y = torch.zeros(300, dtype=torch.float32, device="cuda")
    q.qtt_mlp_forward(m, _f32(X), y)
    torch.cuda.synchronize()
    want, _ = Ln.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), want, rtol=0, atol=2e-6 * max(1.0, np.abs(want).max()))


def test_mlp_gradient_matches_oracle(q):
    import torch
    p = W.mlp_params(8)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (257, Ln.N_FEAT)).astype(np.float32)
    t = rng.uniform(0, 1, 257).astype(np.float32)
    m = q.qtt_mlp_create(p, 512)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.zeros(Ln.N_PARAMS, dtype=torch.float32, device="cuda")
    q.qtt_mlp_grad(m, _f32(X), _f32(t), loss, g)
    torch.cuda.synchronize()
    want_loss, want_g = Ln.mlp_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss.item()) - want_loss) <= 1e-5 * want_loss
    got = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want_g) <= 1e-5 * np.linalg.norm(want_g)
    assert np.abs(got - want_g).max() <= 1e-5 * np.abs(want_g).max()


def test_adam_training_matches_oracle_and_is_deterministic(q):
    import torch
    p0 = W.mlp_params(9)
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (128, Ln.N_FEAT)).astype(np.float32)
    t = (0.3 + 0.2 * np.tanh(X[:, 0] - X[:, 5])).astype(np.float32)
    Xg, tg = _f32(X), _f32(t)
    runs, losses = [], []
    for _ in range(2):
        m = q.qtt_mlp_create(p0, 128)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        ls = []
        for _s in range(30):
            q.qtt_mlp_grad(m, Xg, tg, loss)
            q.qtt_mlp_adam_step(m, 1e-3)
            ls.append(float(loss.item()))
        runs.append(q.qtt_mlp_get_params(m))
        losses.append(ls)
    assert np.array_equal(runs[0], runs[1]) and losses[0] == losses[1]
    assert losses[0][-1] < 0.5 * losses[0][0]
    # the oracle from the same start, in FP64
    p = p0.astype(np.float64)
    mo = np.zeros_like(p)
    vo = np.zeros_like(p)
    for s in range(30):
        _l, g = Ln.mlp_grad(p, X.astype(np.float64), t.astype(np.float64))
        p, mo, vo = Ln.adam_step(p, g, mo, vo, s + 1, 1e-3)
    # Adam normalises each step to ~lr per parameter: FP32 gradient rounding
    # moves a parameter by at most ~lr per step where the gradient is tiny
    assert np.abs(runs[0] - p).max() < 30 * 1e-3 * 0.1
    assert np.linalg.norm(runs[0] - p) < 1e-2 * np.linalg.norm(p - p0)


def test_rank_features_match_oracle(q):
    import torch
    rng = np.random.default_rng(4)
    d, chi, eps, lds = 12, 16, 1e-6, 40
    S = np.zeros((d + 1, lds))
    lens = np.zeros(d + 1, dtype=np.int32)
    ranks = np.zeros(d + 1, dtype=np.int32)
    for k in range(1, d):
        L = int(rng.integers(1, lds + 1))
        s = np.sort(10.0 ** rng.uniform(-12, 0, L))[::-1] * rng.uniform(0.1, 10)
        if k == 5:
            s[:] = 0.0
        S[k, :L] = s
        lens[k] = L
        ranks[k] = O.trunc_rank(s, eps, chi)
    X = torch.zeros((d - 1, Ln.N_FEAT), dtype=torch.float32, device="cuda")
    q.qtt_rank_features(_t(S), torch.as_tensor(lens, device="cuda"), torch.as_tensor(ranks, device="cuda"), d - 1, eps,
                        chi, d, X)
    torch.cuda.synchronize()
    got = X.cpu().numpy()
    for k in range(1, d):
        want = Ln.rank_features(S[k, :lens[k]], int(ranks[k]), eps, chi, k, d)
        np.testing.assert_allclose(got[k - 1], want, rtol=0, atol=1e-6)


@pytest.mark.parametrize("prec", ["fp64"])
def test_learned_round_with_given_proposals_matches_oracle(q, prec):
    """One step from a seeded state with proposals equal to the plain step's
    ranks (and a few deliberately too small), on the same Gaussian sketch:
    the GPU's learned step equals the oracle's learned step, attempt for
    attempt."""
    import torch
    n, chi, eps = 6, 64, 1e-6
    N = 1 << n
    c = W.layered_model(n, 20.0, 5)
    lam2 = (0.5 / c.max()) ** 2
    prev_h = O.tt_round(W.random_tt_cores(2 * n, 20, 1, decay=0.7), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, 20, 2, decay=0.7), 1e-14, chi)
    Lo = O.laplacian_mpo(n, "interleaved", "periodic")
    Co = O.velocity_mps(c, n, "interleaved", 1e-8, 12)
    plain = O.mps_step(Lo, Co, lam2, prev_h, cur_h, eps, chi, (N // 2 + 1, 3), 0.37, n, "interleaved")
    props = [0] + O.mps_ranks(plain)[1:-1] + [0]
    props[6] = max(1, props[6] // 3)  # too small: the check must reject them
    props[7] = max(1, props[7] - 6)
    G = W.gaussian_sketch(11, 512, 256)
    log = []
    want = Ln.mps_step_learned(Lo, Co, lam2, prev_h, cur_h, eps, chi, (N // 2 + 1, 3), 0.37, n, "interleaved", props,
                               G, log=log, p=4)
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, prec=prec, learned=True)
    Gd = _t(G)
    q.qtt_set_rank_model(ctx, None, Gd, oversample=4)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    q.qtt_set_proposals(ctx, props)
    q.qtt_step(L, C, lam2, prev, cur, (N // 2 + 1, 3), 0.37)
    att, acc = q.qtt_learned_stats(ctx)
    assert att == len(log) and acc == sum(ok for _k, _ks, ok in log), (att, acc, log)
    assert 0 < acc < att  # both outcomes occur
    assert q.qtt_mps_ranks(cur) == O.mps_ranks(want)
    assert _rel(_dense(q, cur, N), O.mps_to_dense(want, n, "interleaved")) < 1e-10


def test_step_features_match_the_oracle_spectra(q):
    import torch
    n, chi, eps = 5, 16, 1e-7
    N = 1 << n
    c = W.layered_model(n, 40.0, 11)
    lam2 = (0.5 / c.max()) ** 2
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.15), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.15), 1e-14, chi)
    st = []
    want = O.mps_step(O.laplacian_mpo(n, "interleaved", "periodic"), O.velocity_mps(c, n, "interleaved", 1e-8, 12),
                      lam2, prev_h, cur_h, eps, chi, (N // 2 + 1, 3), 0.37, n, "interleaved", st)
    spec = Ln.round_spectra(st, 2 * n)
    ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=12, eps_c=1e-8, learned=True)
    L = q.qtt_laplacian_mpo(ctx)
    C = q.qtt_velocity_mps(ctx, _t(c))
    prev, cur = q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)
    q.qtt_step(L, C, lam2, prev, cur, (N // 2 + 1, 3), 0.37)
    X = torch.zeros((2 * n - 1, Ln.N_FEAT), dtype=torch.float32, device="cuda")
    q.qtt_step_features(cur, X)
    q.qtt_ctx_sync(ctx)
    got = X.cpu().numpy()
    ranks = O.mps_ranks(want)
    for k in range(1, 2 * n):
        S, r = spec[k]
        assert r == ranks[k]
        f = Ln.rank_features(S, r, eps, chi, k, 2 * n)
        # values at the rounding floor (below 1e-10 sigma_1) differ between any
        # two SVDs; their log features are not compared
        keep = np.ones(Ln.N_FEAT, dtype=bool)
        L = len(S)
        for j in range(Ln.N_SPEC):
            p = (j * (L - 1)) // (Ln.N_SPEC - 1) if L > 1 else 0
            keep[j] = S[p] >= 1e-10 * S[0]
        keep[33] = np.sum(S[r:] ** 2) >= 1e-20 * S[0] ** 2
        np.testing.assert_allclose(got[k - 1][keep], f[keep], rtol=0, atol=2e-6)


def _jacobi_work(q, ctx):
    return q.qtt_profile_read(ctx)["svd_flops"]


def test_trained_network_gains_over_the_plain_round(q):
    """What the trained network gains: a 128x128 layered section (chi = 64,
    eps = 1e-5, FP64) run by the plain solver for 160 steps logs its round
    spectra; the network is trained on them on the GPU (features at step k ->
    rank at step k+1); then 30 further steps are taken three ways from the
    same plain states (teacher-forced): plain rounding, rounding with the
    trained network's proposals, and with the untrained network's.  The
    trained network's rank proposals are far closer to the ranks the rule
    then keeps, and its sketches are accepted where the untrained network's
    are not, while every learned step stays within the rounding rule's
    accuracy of the plain step.  The logged SVD work of the three is printed:
    on this workload most round bonds are within the oversampling margin of
    full rank or capped at chi, so the accepted sketches do not yet pay for
    the rejected ones."""
    import torch
    n, chi, eps = 7, 64, 1e-5
    N = 1 << n
    c = W.layered_model(n, 12.5, 2)
    lam2 = (0.5 / c.max()) ** 2
    dt = 0.5 * 12.5 / c.max()
    t = np.arange(400) * dt
    tau = t - 1.5 / 20.0
    amps = lam2 * (1 - 2 * (np.pi * 20.0 * tau) ** 2) * np.exp(-(np.pi * 20.0 * tau) ** 2)
    src = (N // 2, 2)
    mk = lambda: q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=32, eps_c=1e-8, learned=True)
    ctx_p = mk()
    L = q.qtt_laplacian_mpo(ctx_p)
    C = q.qtt_velocity_mps(ctx_p, _t(c))
    prev, cur = q.qtt_mps_create_zero(ctx_p), q.qtt_mps_create_zero(ctx_p)
    K = 160
    feats, ranks = [], []
    X = torch.zeros((2 * n - 1, Ln.N_FEAT), dtype=torch.float32, device="cuda")
    for k in range(K):
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        q.qtt_step_features(cur, X)
        q.qtt_ctx_sync(ctx_p)
        feats.append(X.cpu().numpy().copy())
        ranks.append(q.qtt_mps_ranks(cur))
    Xs = np.concatenate(feats[:-1])
    ys = np.concatenate([np.array(r[1:-1], dtype=np.float32) / chi for r in ranks[1:]])
    p0 = W.mlp_params(7)
    trained = q.qtt_mlp_create(p0, len(Xs))
    untrained = q.qtt_mlp_create(p0, len(Xs))
    Xg, yg = _f32(Xs), _f32(ys)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    q.qtt_mlp_grad(trained, Xg, yg, loss)
    loss0 = float(loss.item())
    for _ in range(600):
        q.qtt_mlp_grad(trained, Xg, yg, loss)
        q.qtt_mlp_adam_step(trained, 2e-3)
    assert float(loss.item()) < 0.05 * loss0
    G = _t(W.gaussian_sketch(11, 1 << n, 160))
    ctx_t, ctx_u = mk(), mk()
    q.qtt_set_rank_model(ctx_t, trained, G)
    q.qtt_set_rank_model(ctx_u, untrained, G)
    Lt, Ct = q.qtt_laplacian_mpo(ctx_t), q.qtt_velocity_mps(ctx_t, _t(c))
    Lu, Cu = q.qtt_laplacian_mpo(ctx_u), q.qtt_velocity_mps(ctx_u, _t(c))
    for x in (ctx_p, ctx_t, ctx_u):
        q.qtt_profile_start(x, timing=False, log_svd=True)
    worst = 0.0
    err = {"t": [], "u": []}
    last = None
    for k in range(K, K + 30):
        ph, chh = q.qtt_mps_get_cores(prev), q.qtt_mps_get_cores(cur)
        outs, props = [], []
        for ctx, Lx, Cx in ((ctx_t, Lt, Ct), (ctx_u, Lu, Cu)):
            a, b = q.qtt_mps_from_cores(ctx, ph), q.qtt_mps_from_cores(ctx, chh)
            q.qtt_step(Lx, Cx, lam2, a, b, src, float(amps[k]))
            outs.append(_dense(q, b, N))
            props.append(q.qtt_get_proposals(ctx))
        q.qtt_step(L, C, lam2, prev, cur, src, float(amps[k]))
        ref = _dense(q, cur, N)
        worst = max(worst, _rel(outs[0], ref), _rel(outs[1], ref))
        r = q.qtt_mps_ranks(cur)
        if last is not None:
            err["t"].append(np.mean(np.abs(np.array(last[0][1:-1]) - np.array(r[1:-1]))))
            err["u"].append(np.mean(np.abs(np.array(last[1][1:-1]) - np.array(r[1:-1]))))
        last = props
    at_t, ac_t = q.qtt_learned_stats(ctx_t)
    at_u, ac_u = q.qtt_learned_stats(ctx_u)
    w_p, w_t, w_u = _jacobi_work(q, ctx_p), _jacobi_work(q, ctx_t), _jacobi_work(q, ctx_u)
    et, eu = float(np.mean(err["t"])), float(np.mean(err["u"]))
    print(f"\nlearned rounding, 30 steps: mean |proposal - kept rank| trained {et:.2f}, untrained {eu:.2f}; "
          f"trained {ac_t}/{at_t} sketches accepted, untrained {ac_u}/{at_u}; "
          f"Jacobi work vs plain: trained {w_t / w_p:.3f}, untrained {w_u / w_p:.3f}; worst step difference {worst:.2e}")
    assert et < 0.25 * eu
    assert ac_t > 0 and ac_t / max(at_t, 1) > ac_u / max(at_u, 1)
    assert worst < 1e-4
