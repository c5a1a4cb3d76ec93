"""The truncated MPS dynamics is chaotic once the chi cap binds.

This is why long runs are compared step by step (teacher-forced) and not as
free-running trajectories: the oracle against itself, with one source sample
changed by one part in 1e15 (a relative change below FP64 rounding of most
operations), separates by O(1) within 150 steps of the 64 x 64 workload
(chi = 32 binds from step ~40), while with a cap that does not bind
(chi = 64 = the largest rank the 12-site grid allows, eps = 1e-14) the same
change stays below 1e-6.  Eq. 2 is linear, so the exponential growth comes
from the truncation decisions of Sec. 4.3 alone."""
import numpy as np

from oracle import qtt_oracle as O
import workloads as W


def _separation(chi, eps, steps, checks):
    wl = W.config(0)
    n, N = wl.n, wl.N
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = np.array(wl.source_amplitudes(c), dtype=np.float64)
    amps2 = amps.copy()
    amps2[20] *= 1.0 + 1e-15
    assert amps2[20] != amps[20]
    Lo = O.laplacian_mpo(n, wl.order, wl.bc)
    Co = O.velocity_mps(c, n, wl.order, wl.eps_c, wl.chi_c)
    src = (N // 2 + 1, N // 2)
    a = [O.zero_mps(2 * n), O.zero_mps(2 * n)]
    b = [O.zero_mps(2 * n), O.zero_mps(2 * n)]
    out = {}
    for k in range(steps):
        a = [a[1], O.mps_step(Lo, Co, lam2, a[0], a[1], eps, chi, src, float(amps[k]), n, wl.order)]
        b = [b[1], O.mps_step(Lo, Co, lam2, b[0], b[1], eps, chi, src, float(amps2[k]), n, wl.order)]
        if k + 1 in checks:
            da, db = O.mps_to_dense(a[1], n, wl.order), O.mps_to_dense(b[1], n, wl.order)
            out[k + 1] = float(np.linalg.norm(da - db) / np.linalg.norm(da))
    return out


def test_a_1e15_change_of_one_source_sample_grows_to_order_one_once_the_cap_binds():
    wl = W.config(0)
    sep = _separation(wl.chi, wl.eps, 150, {60, 100, 150})
    assert sep[60] < 1e-11, sep
    assert sep[100] > 1e-3, sep
    assert sep[150] > 0.1, sep


def test_the_same_change_stays_small_when_the_cap_does_not_bind():
    sep = _separation(64, 1e-14, 150, {150})
    assert sep[150] < 1e-6, sep
