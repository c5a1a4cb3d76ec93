"""Pins of the learned-rank oracles (oracle/learned.py, numpy, and the
learned form of the C++ oracle, oracle/cxx_learned.py) against mathematics
that does not come from either oracle: central finite differences,
hand-built networks, Adam's closed-form first step, a spectrum whose
features are known in closed form, exactly low-rank matrices, and brute-force
SVDs for the range finder's acceptance guarantees.  Every pin runs on both
oracles; the last tests compare them with each other."""
import numpy as np
import pytest

from oracle import cxx
from oracle import cxx_learned
from oracle import learned
from oracle import qtt_oracle as O
import workloads as W

IMPLS = {"numpy": (learned, O), "cxx": (cxx_learned, cxx)}


@pytest.fixture(params=sorted(IMPLS))
def impl(request):
    """(learned-form oracle, plain oracle of the same implementation)."""
    return IMPLS[request.param]


def test_mlp_gradient_matches_central_differences(impl):
    Ln, _ = impl
    rng = np.random.default_rng(3)
    p = W.mlp_params(5).astype(np.float64)
    p += 0.05 * rng.standard_normal(p.shape)  # nonzero biases too
    X = rng.standard_normal((6, Ln.N_FEAT))
    t = rng.uniform(0, 1, 6)
    _, g = Ln.mlp_grad(p, X, t)
    idx = np.concatenate([rng.choice(Ln.N_PARAMS - 129, 300, replace=False), np.arange(Ln.N_PARAMS - 129, Ln.N_PARAMS)])
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (Ln.mse_loss(Ln.mlp_forward(pp, X)[0], t) - Ln.mse_loss(Ln.mlp_forward(pm, X)[0], t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def _hand_network(Ln):
    """y = relu(x0) + relu(-x0) + 0.25 = |x0| + 0.25"""
    W1 = np.zeros((Ln.WIDTH, Ln.N_FEAT))
    W1[0, 0], W1[1, 0] = 1.0, -1.0
    W2 = np.eye(Ln.WIDTH)
    W3 = np.zeros((1, Ln.WIDTH))
    W3[0, :2] = 1.0
    return Ln.pack([W1, np.zeros(Ln.WIDTH), W2, np.zeros(Ln.WIDTH), W3, [0.25]])


def test_mlp_forward_and_gradient_of_a_hand_built_network(impl):
    Ln, _ = impl
    p = _hand_network(Ln)
    X = np.zeros((2, Ln.N_FEAT))
    X[0, 0], X[1, 0] = 0.3, -0.7
    y, _ = Ln.mlp_forward(p, X)
    np.testing.assert_allclose(y, [0.55, 0.95], rtol=0, atol=1e-15)
    t = np.array([0.5, 1.0])
    loss, g = Ln.mlp_grad(p, X, t)
    assert abs(loss - ((0.05 ** 2 + 0.05 ** 2) / 2)) < 1e-15
    gW1, gb1, gW2, gb2, gW3, gb3 = Ln.unpack(g)
    # dL/dy = 2 (y - t) / n = [0.05, -0.05]
    assert abs(gb3[0] - 0.0) < 1e-15
    # dL/dW1[0,0] = 0.05 * 1 * x0 (only sample 0 activates unit 0) = 0.015
    assert abs(gW1[0, 0] - 0.015) < 1e-15
    # unit 1 (a = -x0) is active for sample 1 only: dL/dW1[1,0] = -0.05 * x0 = 0.035
    assert abs(gW1[1, 0] - 0.035) < 1e-15
    assert abs(gW3[0, 0] - 0.05 * 0.3) < 1e-15 and abs(gW3[0, 1] - (-0.05 * 0.7)) < 1e-15


def test_adam_first_steps_closed_form(impl):
    Ln, _ = impl
    p0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    m = v = np.zeros(3)
    p1, m, v = Ln.adam_step(p0, g, m, v, 1, lr=1e-2)
    np.testing.assert_allclose(p1, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # with a constant gradient the bias-corrected moments stay g and g^2
    p2, m, v = Ln.adam_step(p1, g, m, v, 2, lr=1e-2)
    np.testing.assert_allclose(p2, p1 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_rank_features_of_a_geometric_spectrum(impl):
    Ln, _ = impl
    S = 10.0 ** (-np.arange(64) / 8.0)
    f = Ln.rank_features(S, 20, 1e-4, 32, 3, 10)
    for j in range(32):
        p = (j * 63) // 31
        assert abs(f[j] - (-p / 8.0) / 16.0) < 1e-14
    assert f[32] == 20 / 32
    disc = np.sum(10.0 ** (-np.arange(20, 64) / 4.0))
    assert abs(f[33] - np.log10(disc) / 32.0) < 1e-14
    assert abs(f[34] - (-4 / 16.0)) < 1e-15
    assert f[35] == 3 / 10 and f[36] == 8 / 32
    assert f[37] == 33 / 32  # 10^(-i/8) >= 1e-4 for i <= 32
    assert f[38] == 64 / 64 and f[39] == 1.0
    z = Ln.rank_features(np.zeros(5), 1, 1e-6, 16, 2, 8)
    assert np.all(z[:32] == -1.0) and z[33] == -1.0 and z[37] == 0.0


def test_propose_rank_rounds_up_and_clamps(impl):
    Ln, _ = impl
    assert Ln.propose_rank(0.5, 64) == 32
    assert Ln.propose_rank(0.5001, 64) == 33
    assert Ln.propose_rank(-3.0, 64) == 1
    assert Ln.propose_rank(7.0, 64) == 64


def _with_spectrum(rng, l, m, s):
    U, _ = np.linalg.qr(rng.standard_normal((l, len(s))))
    V, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    return (U * s) @ V.T


def test_range_finder_is_exact_on_a_low_rank_matrix(impl):
    Ln, _ = impl
    rng = np.random.default_rng(1)
    s = np.array([5.0, 2.0, 1.0, 0.5, 0.1])
    X = _with_spectrum(rng, 40, 30, s)
    G = W.gaussian_sketch(2, 40, 12)
    ok, r, Vt, US, Sb, rho = Ln.range_finder_svd(X, G, 1e-10, 20)
    assert ok and r == 5 and rho < 1e-13
    np.testing.assert_allclose(Sb[:5], s, rtol=0, atol=1e-13)
    np.testing.assert_allclose(US @ Vt, X, rtol=0, atol=1e-13)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(5), atol=1e-13)


def test_range_finder_acceptance_guarantees_against_brute_force(impl):
    """Whenever the check accepts: uncapped cuts leave no discarded direction
    above sqrt(2) eps sigma_1; capped cuts stay within (1+tau)^2 of the
    optimal discarded weight.  Both outcomes occur."""
    Ln, _ = impl
    rng = np.random.default_rng(9)
    seen = {"acc_unc": 0, "acc_cap": 0, "rej": 0}
    for trial in range(120):
        l, m = int(rng.integers(30, 90)), int(rng.integers(30, 90))
        n = min(l, m)
        rate = rng.uniform(0.05, 1.5)
        s = np.exp(-rate * np.arange(n)) * rng.uniform(0.5, 2.0)
        X = _with_spectrum(rng, l, m, s)
        eps = 10.0 ** rng.uniform(-9, -2)
        chi = int(rng.integers(2, n))
        ks = int(rng.integers(3, n))
        G = W.gaussian_sketch(100 + trial, l, ks)
        ok, r, Vt, US, Sb, rho = Ln.range_finder_svd(X, G, eps, chi)
        sx = np.linalg.svd(X, compute_uv=False)
        if not ok:
            seen["rej"] += 1
            continue
        proj = Vt.T @ Vt
        E = X - X @ proj
        c = int(np.count_nonzero(Sb >= eps * Sb[0]))
        if c < chi:
            seen["acc_unc"] += 1
            assert np.linalg.norm(E, 2) <= np.sqrt(2.0) * eps * sx[0] * (1 + 1e-9) + 1e-14
        else:
            seen["acc_cap"] += 1
            opt = np.sum(sx[chi:] ** 2)
            assert np.sum(E * E) <= (1 + Ln.TAU) ** 2 * opt * (1 + 1e-9) + 1e-26
    assert all(v > 0 for v in seen.values()), seen


def test_acceptance_keeps_its_guarantees_on_narrow_sketches(impl):
    """Sketches only 1-5 wider than chi, which often miss part of the top
    chi directions, with eps = 1e-12 (both capped and uncapped cuts occur):
    every accepted sketch keeps its guarantee (capped: discarded weight
    within (1+tau)^2 of the optimal tail; uncapped: no discarded direction
    above sqrt(2) eps sigma_1), and capped acceptances and rejections both
    occur often."""
    Ln, _ = impl
    rng = np.random.default_rng(42)
    cap = unc = rej = 0
    for trial in range(200):
        l, m = int(rng.integers(30, 60)), int(rng.integers(30, 60))
        n = min(l, m)
        chi = int(rng.integers(3, n // 2))
        ks = chi + int(rng.integers(1, 6))
        X = _with_spectrum(rng, l, m, np.exp(-rng.uniform(0.3, 3.0) * np.arange(n)))
        eps = 1e-12
        ok, r, Vt, US, Sb, rho = Ln.range_finder_svd(X, W.gaussian_sketch(500 + trial, l, ks), eps, chi)
        if not ok:
            rej += 1
            continue
        E = X - X @ (Vt.T @ Vt)
        sx = np.linalg.svd(X, compute_uv=False)
        if int(np.count_nonzero(Sb >= eps * Sb[0])) < chi:
            unc += 1
            assert np.linalg.norm(E, 2) <= np.sqrt(2.0) * eps * sx[0] * (1 + 1e-9) + 1e-14, trial
        else:
            cap += 1
            assert np.sum(E * E) <= (1 + Ln.TAU) ** 2 * np.sum(sx[chi:] ** 2) * (1 + 1e-9) + 1e-26, trial
    assert cap > 20 and rej > 20, (cap, unc, rej)


def test_learned_round_without_proposals_is_the_plain_round(impl):
    Ln, P = impl
    cores = W.random_tt_cores(10, 16, 4, decay=0.2)
    G = W.gaussian_sketch(3, 64, 64)
    a = P.tt_round(cores, 1e-6, 8)
    b = Ln.tt_round_learned(cores, 1e-6, 8, None, G)
    assert O.mps_ranks(a) == O.mps_ranks(b)
    np.testing.assert_allclose(O.mps_full(b), O.mps_full(a), rtol=0, atol=1e-14 * np.abs(O.mps_full(a)).max())


def test_learned_round_with_exact_proposals_accepts_and_matches(impl):
    """A state of exact bond ranks 3 (below the cap) padded to rank 12: the
    proposals equal the true ranks, every sketch (width 3 + 2) sees the cut
    and is accepted, and the result equals the plain round's."""
    Ln, P = impl
    rng = np.random.default_rng(5)
    d = 14
    small = [rng.standard_normal((1 if k == 0 else 3, 2, 1 if k == d - 1 else 3)) for k in range(d)]
    doubled = O.mps_sum([(0.5, small), (0.5, small), (1.0, small), (-1.0, small)])
    G = W.gaussian_sketch(6, 64, 64)
    props = [0] + [3] * (d - 1)
    log = []
    b = Ln.tt_round_learned(doubled, 1e-10, 16, props, G, p=2, log=log)
    a = P.tt_round(doubled, 1e-10, 16)
    assert O.mps_ranks(b) == O.mps_ranks(a)
    assert len(log) >= 4 and all(ok for _k, _ks, ok in log), log
    fa = O.mps_full(a)
    np.testing.assert_allclose(O.mps_full(b), fa, rtol=0, atol=1e-12 * np.abs(fa).max())


# ---------------------------------------------------------------------------
# the two learned-form oracles against each other
# ---------------------------------------------------------------------------
def test_learned_forms_agree_on_features_network_and_range_finder():
    assert cxx_learned.param_count() == cxx_learned.N_PARAMS == learned.N_PARAMS
    rng = np.random.default_rng(21)
    p = W.mlp_params(7).astype(np.float64) + 0.05 * rng.standard_normal(learned.N_PARAMS)
    Xf = rng.standard_normal((9, learned.N_FEAT))
    t = rng.uniform(0, 1, 9)
    np.testing.assert_allclose(cxx_learned.mlp_forward(p, Xf)[0], learned.mlp_forward(p, Xf)[0], rtol=0, atol=1e-13)
    (la, ga), (lb, gb) = cxx_learned.mlp_grad(p, Xf, t), learned.mlp_grad(p, Xf, t)
    assert abs(la - lb) < 1e-13
    np.testing.assert_allclose(ga, gb, rtol=0, atol=1e-13)
    for L, r, eps, chi in ((50, 12, 1e-6, 16), (7, 7, 1e-3, 64), (300, 128, 1e-8, 128)):
        S = np.sort(10.0 ** rng.uniform(-12, 0, L))[::-1]
        np.testing.assert_allclose(cxx_learned.rank_features(S, r, eps, chi, 5, 20),
                                   learned.rank_features(S, r, eps, chi, 5, 20), rtol=0, atol=1e-15)
    for trial in range(20):
        l, m = int(rng.integers(20, 70)), int(rng.integers(20, 70))
        s = np.exp(-rng.uniform(0.05, 1.0) * np.arange(min(l, m)))
        Xm = _with_spectrum(rng, l, m, s)
        eps, chi, ks = 10.0 ** rng.uniform(-8, -2), int(rng.integers(2, min(l, m))), int(rng.integers(3, min(l, m)))
        G = W.gaussian_sketch(300 + trial, l, ks)
        a, b = cxx_learned.range_finder_svd(Xm, G, eps, chi), learned.range_finder_svd(Xm, G, eps, chi)
        assert a[0] == b[0] and a[1] == b[1]
        np.testing.assert_allclose(a[4], b[4], rtol=0, atol=1e-13 * b[4][0])
        assert abs(a[5] - b[5]) <= 1e-12 * max(1.0, b[5])
        np.testing.assert_allclose(a[3] @ a[2], b[3] @ b[2], rtol=0, atol=1e-12)


def test_learned_rounds_agree_with_proposals_accepted_and_rejected():
    """Proposals equal to the plain round's ranks on odd bonds (accepted) and
    a third of them on even bonds (rejected, full SVD): both oracles make the
    same decisions and the same rounded state.  The sketch multiplies the
    bond's left index by a fixed Gaussian matrix, so this needs both QR
    sweeps to leave the bonds in the same gauge, which they do."""
    cores = O.tt_round(W.random_tt_cores(12, 32, 8, decay=0.5), 1e-14, 32)
    th = O.mps_sum([(1.0, cores), (0.3, O.tt_round(W.random_tt_cores(12, 32, 9, decay=0.5), 1e-14, 32))])
    G = W.gaussian_sketch(11, 128, 128)
    rk = O.mps_ranks(O.tt_round(th, 1e-4, 24))
    props = [0] + [rk[k] if k % 2 else max(1, rk[k] // 3) for k in range(1, 12)]
    la, lb = [], []
    a = cxx_learned.tt_round_learned(th, 1e-4, 24, props, G, p=8, log=la)
    b = learned.tt_round_learned(th, 1e-4, 24, props, G, p=8, log=lb)
    assert la == lb and any(ok for _k, _ks, ok in lb) and not all(ok for _k, _ks, ok in lb), lb
    assert O.mps_ranks(a) == O.mps_ranks(b)
    fb = O.mps_full(b)
    np.testing.assert_allclose(O.mps_full(a), fb, rtol=0, atol=1e-12 * np.abs(fb).max())
