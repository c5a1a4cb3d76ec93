"""Tolerances of the reduced-precision forms (FP32 and 3xTF32 contractions),
shared by the GPU parity tests.

A step of these forms perturbs every bond matrix by about u = 1e-7 of its
norm (FP32 rounding of the contractions and QR, accumulated over the step's
dependent factorisations).  Where a cut discards values, the kept subspace
then turns by about u sigma_1 / (sigma_r - sigma_{r+1}), and the truncated
matrix, whose discarded and kept directions near the cut carry about
sigma_r, moves by u sigma_r / (sigma_r - sigma_{r+1}) of the state's norm.
So with h the smallest relative gap (sigma_r - sigma_{r+1}) / sigma_r over
the discarding cuts of a step (from the oracle's spectra), one step from a
shared state is held to

    err <= min(2e-5 + 1e-6 / h, 1e-4)      (relative L2 of the dense field)

and a step with h < 1e-4 (a gap within a few FP32 roundings of the values
at the cut) is a cut that FP32 cannot resolve ("degenerate at FP32
resolution", Sec. 4.3 gives no rule for ties): it is reported and counted,
not held to a bound.

Below eps = 1e-6 the cuts themselves sit under the FP32 resolution of the
step (u ~ 6e-8 times its growth hides singular values below ~1e-6 sigma_1,
and rank decisions there follow rounding, not the spectrum): the forms are
stated for eps >= 1e-6, and at smaller eps a step is held to the workloads'
accuracy target, 1e-3 relative L2.

Ranks: FP32 rounding moves every singular value by up to about 1e-6 sigma_1
(u times the growth over the step), so a value within 1e-6 sigma_1 of the
threshold eps sigma_1 may fall on either side of it: at each bond the ranks
may differ by 2 plus the number of the oracle's values in that band.  Below
eps = 1e-6 the threshold itself is under that resolution and the kept rank
follows rounding: only the cap is checked (no rank above chi)."""
import numpy as np

DEGENERATE_H = 1e-4
TOL_BASE, TOL_GAP, TOL_CAP = 2e-5, 1e-6, 1e-4
RANK_BAND = 1e-6
FP32_RESOLUTION = 1e-6  # smallest eps whose cuts the FP32 forms resolve
TOL_BELOW_RESOLUTION = 1e-3


def gaps(stats):
    """(g, h): smallest gap at a discarding cut relative to sigma_1 and to sigma_r."""
    g = h = 1.0
    for _kind, _k, S, r in stats:
        if r < len(S) and S[0] > 0 and S[r - 1] > 0:
            d = max(S[r - 1] - S[r], 1e-300)
            g = min(g, d / S[0])
            h = min(h, d / S[r - 1])
    return g, h


def tol32(stats, eps):
    """(tolerance, degenerate) of one step of the FP32 / 3xTF32 forms."""
    _g, h = gaps(stats)
    if eps < FP32_RESOLUTION:
        return TOL_BELOW_RESOLUTION, False
    return min(TOL_BASE + TOL_GAP / h, TOL_CAP), h < DEGENERATE_H


def rank_allowance(stats, eps, d):
    """Allowed |rank difference| at bonds 0..d (from the round's spectra)."""
    allow = [0] * (d + 1)
    for kind, k, S, _r in stats:
        if kind != "round" or len(S) == 0 or S[0] <= 0:
            continue
        lo, hi = eps * S[0] - RANK_BAND * S[0], eps * S[0] + RANK_BAND * S[0]
        band = int(np.count_nonzero((S >= lo) & (S <= hi)))
        allow[k] = 2 + band
    return allow


def ranks_ok(got, want, stats, eps, chi=None):
    if eps < FP32_RESOLUTION:
        return chi is None or max(got) <= chi
    allow = rank_allowance(stats, eps, len(want) - 1)
    return all(abs(a - b) <= max(al, 0) for a, b, al in zip(got, want, allow))
