"""FP64 CPU oracle of the learned rank proposal and the randomised rounding.

TEST INFRASTRUCTURE ONLY, like ``qtt_oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code with the CUDA library.

The paper rounds every bond with a full SVD (Sec. 4.3).  The learned form
keeps that rule as the arbiter and only changes how the kept subspace is found:

* a small MLP (3 linear layers, width 128, ReLU, FP32 parameters) reads 40
  features of a bond's singular-value spectrum at step k and proposes the
  bond's rank at step k+1 (the proposal is chi * output, rounded up);
* the round's SVD of that bond at step k+1 then uses a randomised range
  finder of width r_hat + p (p = 16) (Halko, Martinsson & Tropp, SIAM Review 2011,
  Algorithm 4.1 followed by the direct SVD of Sec. 5.1): Y = X^T Omega,
  Q = qr(Y), B = Q^T X^T, SVD of B;
* an exact check decides whether the sketch is good enough for the Sec. 4.3
  rule (``range_finder_svd``); if not, the bond falls back to the full SVD.

Training: mean squared error on the scaled rank, Adam (Kingma & Ba, ICLR 2015,
Algorithm 1).  Parameters and the Gaussian test matrix come from the seeded
generators in ``workloads`` (inputs, not arithmetic of the method).

Every function is pinned by ``tests/test_oracle_learned.py``.
"""
from __future__ import annotations

import numpy as np

from oracle import qtt_oracle as O

N_FEAT = 40
WIDTH = 128
N_SPEC = 32  # spectrum samples among the features
OVERSAMPLE = 16
TAU = 0.05

# flat parameter layout: W1 (WIDTH x N_FEAT), b1, W2 (WIDTH x WIDTH), b2, W3 (1 x WIDTH), b3
SHAPES = [(WIDTH, N_FEAT), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (1, WIDTH), (1,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(flat: np.ndarray) -> list[np.ndarray]:
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def pack(parts: list[np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


# ---------------------------------------------------------------------------
# Features of one bond's spectrum
# ---------------------------------------------------------------------------
def rank_features(S: np.ndarray, r: int, eps: float, chi: int, k: int, d: int) -> np.ndarray:
    """40 features of bond k (of d sites) after a truncation that kept r of
    the descending singular values S (threshold eps, cap chi):

    0..31  log10(S_p / S_0) at 32 evenly spaced positions p = floor(j (L-1) / 31)
           of the L values, clipped to [-16, 0] and divided by 16
           (-1 everywhere when S_0 = 0);
    32     r / chi;
    33     log10(discarded weight / S_0^2), clipped to [-32, 0], divided by 32
           (-1 when S_0 = 0 or nothing is discarded);
    34     log10(eps) / 16;
    35     k / d;
    36     min(2^k, 2^(d-k), chi) / chi;
    37     #{S_i >= eps S_0} / chi;
    38     L / (2 chi);
    39     1."""
    S = np.asarray(S, dtype=np.float64)
    L = len(S)
    f = np.zeros(N_FEAT)
    s0 = S[0] if L else 0.0
    for j in range(N_SPEC):
        p = (j * (L - 1)) // (N_SPEC - 1) if L > 1 else 0
        if s0 > 0 and S[p] > 0:
            f[j] = min(max(np.log10(S[p] / s0), -16.0), 0.0) / 16.0
        else:
            f[j] = -1.0
    f[32] = r / chi
    disc = float(np.sum(S[r:] ** 2)) if L else 0.0
    f[33] = (min(max(np.log10(disc / (s0 * s0)), -32.0), 0.0) / 32.0) if (s0 > 0 and disc > 0) else -1.0
    f[34] = np.log10(eps) / 16.0 if eps > 0 else -1.0
    f[35] = k / d
    f[36] = min(2 ** k, 2 ** (d - k), chi) / chi
    f[37] = (int(np.count_nonzero(S >= eps * s0)) if s0 > 0 else 0) / chi
    f[38] = L / (2.0 * chi)
    f[39] = 1.0
    return f


# ---------------------------------------------------------------------------
# MLP: forward, loss, backward, Adam
# ---------------------------------------------------------------------------
def mlp_forward(params: np.ndarray, X: np.ndarray) -> tuple[np.ndarray, dict]:
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = (h2 @ W3.T + b3)[:, 0]
    return y, {"X": X, "a1": a1, "h1": h1, "a2": a2, "h2": h2}


def mse_loss(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((np.asarray(y) - np.asarray(t)) ** 2))


def mlp_grad(params: np.ndarray, X: np.ndarray, t: np.ndarray) -> tuple[float, np.ndarray]:
    """Loss (mean squared error) and its gradient with respect to every
    parameter, by the chain rule through the three layers."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    y, c = mlp_forward(params, X)
    n = len(y)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n  # dL/dy
    gW3 = dy[None, :] @ c["h2"]
    gb3 = np.array([dy.sum()])
    dh2 = dy[:, None] @ W3
    da2 = dh2 * (c["a2"] > 0)
    gW2 = da2.T @ c["h1"]
    gb2 = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (c["a1"] > 0)
    gW1 = da1.T @ c["X"]
    gb1 = da1.sum(0)
    return mse_loss(y, t), pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(params, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1); t counts from 1.
    Returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def propose_rank(y: float, chi: int) -> int:
    """r_hat = ceil(chi * y), clamped to [1, chi]."""
    return int(min(max(int(np.ceil(chi * y)), 1), chi))


# ---------------------------------------------------------------------------
# Randomised range finder with the exact acceptance check
# ---------------------------------------------------------------------------
def range_finder_svd(X: np.ndarray, Omega: np.ndarray, eps: float, chi: int, tau: float = TAU):
    """Truncated SVD of X (l x m) for the Sec. 4.3 rule from a sketch of its
    row space.  Omega (l x ks) is Gaussian.

        Y = X^T Omega,  Q = qr(Y) (m x ks),  B = Q^T X^T = (X Q)^T,
        B = Ub diag(Sb) Vb^T,  X ~ Vb diag(Sb) (Q Ub)^T,
        rho = ||X - X Q Q^T||_F, computed explicitly.

    Acceptance, with c = #{Sb_i >= eps Sb_0}:
      c >= ks: reject (the cut is not inside the sketch);
      c <  chi (uncapped): accept iff rho <= eps Sb_0; every discarded
               direction then has a singular value <= sqrt(2) eps sigma_1
               (Weyl on X X^T = A A^T + E E^T below: sigma_{r+1}(X)^2 <=
               Sb_{r+1}^2 + rho^2);
      c >= chi (capped at chi): accept iff
               rho^2 <= ((1+tau)^2 - 1) sum_{i>=chi} Sb_i^2.
               Why: X X^T = A A^T + E E^T with A = X Q Q^T and E = X - A
               (A E^T = 0), so by Ky Fan's maximum principle
               sum_{i<chi} sigma_i(X)^2 <= sum_{i<chi} Sb_i^2 + ||E||_F^2 and
               the optimal tail ||X||^2 - sum_{i<chi} sigma_i(X)^2 is at
               least sum_{i>=chi} Sb_i^2; the sketch's discarded weight is
               sum_{i>=chi} Sb_i^2 + rho^2, hence within (1+tau)^2 of the
               optimum.  (Bounding each sigma_i(X) <= Sb_i + rho instead, by
               Weyl, leaves a cross term 2 rho sum Sb_i that exceeds the tail
               on every realistic bond, so that form never accepts.)
    Returns (accepted, r, Vt (r x m), US (l x r), Sb, rho)."""
    X = np.asarray(X, dtype=np.float64)
    Y = X.T @ Omega
    Q, _ = np.linalg.qr(Y)
    B = Q.T @ X.T
    Ub, Sb, Vbt = np.linalg.svd(B, full_matrices=False)
    E = X - (X @ Q) @ Q.T
    rho = float(np.sqrt(np.sum(E * E)))
    ks = Omega.shape[1]
    s0 = Sb[0] if len(Sb) else 0.0
    c = int(np.count_nonzero(Sb >= eps * s0)) if s0 > 0 else 0
    r = O.trunc_rank(Sb, eps, chi)
    if s0 == 0.0:
        accepted = rho == 0.0
    elif c >= ks:
        accepted = False
    elif c < chi:
        accepted = rho <= eps * s0
    else:
        accepted = rho * rho <= ((1.0 + tau) ** 2 - 1.0) * float(np.sum(Sb[chi:] ** 2))
    Vt = (Q @ Ub[:, :r]).T
    US = Vbt[:r].T * Sb[:r]
    return accepted, r, Vt, US, Sb, rho


def tt_round_learned(A: list[np.ndarray], eps: float, chi: int, proposals, G: np.ndarray,
                     p: int = OVERSAMPLE, tau: float = TAU, stats: list | None = None,
                     log: list | None = None) -> list[np.ndarray]:
    """tt_round (Sec. 4.3) where bond k of the SVD sweep first tries the range
    finder of width ks = proposals[k] + p with Omega = G[:l, :ks] (the
    top-left block of one fixed Gaussian matrix), when ks < min(l, 2 r);
    rejected or unproposed bonds take the full SVD.  log receives
    (k, ks, accepted) per attempt."""
    A = [np.array(c, dtype=np.float64) for c in A]
    d = len(A)
    for k in range(d - 1):
        l, _, r = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(l * 2, r))
        A[k] = Q.reshape(l, 2, Q.shape[1])
        A[k + 1] = np.einsum("ij,jsk->isk", R, A[k + 1])
    for k in range(d - 1, 0, -1):
        l, _, r = A[k].shape
        X = A[k].reshape(l, 2 * r)
        done = False
        ph = proposals[k] if proposals is not None else 0
        if ph > 0:
            ks = ph + p
            if ks < min(l, 2 * r):
                ok, rr, Vt, US, Sb, _rho = range_finder_svd(X, G[:l, :ks], eps, chi, tau)
                if log is not None:
                    log.append((k, ks, ok))
                if ok:
                    if stats is not None:
                        stats.append(("round_rf", k, Sb.copy(), rr))
                    A[k] = Vt.reshape(rr, 2, r)
                    A[k - 1] = np.einsum("isj,jk->isk", A[k - 1], US)
                    done = True
        if not done:
            U, S, Vt = O._svd(X)
            rr = O.trunc_rank(S, eps, chi)
            if stats is not None:
                stats.append(("round", k, S.copy(), rr))
            A[k] = Vt[:rr].reshape(rr, 2, r)
            A[k - 1] = np.einsum("isj,jk->isk", A[k - 1], U[:, :rr] * S[:rr])
    return A


def mps_step_learned(L, c2, lambda2, prev, cur, eps, chi, src, amp, n, order, proposals, G,
                     stats=None, log=None, p: int = OVERSAMPLE, tau: float = TAU):
    """Eq. 17 step whose round uses tt_round_learned."""
    phi = O.zipup_lr(L, cur, eps, chi, stats)
    eta = O.zipup_rl(O.diagonal_mpo(c2), phi, eps, chi, stats)
    terms = [(2.0, cur), (-1.0, prev), (lambda2, eta)]
    if src is not None:
        terms.append((amp, O.product_state(src[0], src[1], n, order)))
    return tt_round_learned(O.mps_sum(terms), eps, chi, proposals, G, p=p, tau=tau, stats=stats, log=log)


def round_spectra(stats: list, d: int) -> dict:
    """Bond k -> (S, r) of the round's SVD sweep, from a stats list."""
    out = {}
    for kind, k, S, r in stats:
        if kind in ("round", "round_rf"):
            out[k] = (S, r)
    return out
