"""The tolerance rules of the reduced-precision forms (tests/fp32_bounds.py),
on hand-made spectra: the gaps they read, the ceiling no tolerance passes,
the degenerate-cut flag, and the rank allowance around the Sec. 4.3
threshold."""
import numpy as np
import pytest

from fp32_bounds import (DEGENERATE_H, FP32_RESOLUTION, TOL_BASE, TOL_CAP, TOL_GAP, gaps, rank_allowance, ranks_ok,
                         tol32)


def _stat(kind, k, S, r):
    return (kind, k, np.asarray(S, dtype=float), r)


def test_gaps_read_the_discarding_cuts_only():
    stats = [
        _stat("round", 1, [4.0, 2.0, 1.0, 0.5], 2),  # cut between 2.0 and 1.0: g = 1/4, h = 1/2
        _stat("zip_lr", 2, [1.0, 0.9, 0.899], 2),  # cut between 0.9 and 0.899: g = 1e-3, h = 1.1e-3
        _stat("round", 3, [3.0, 1.0], 2),  # keeps everything: no cut
        _stat("round", 4, [0.0, 0.0], 1),  # zero matrix: no cut
    ]
    g, h = gaps(stats)
    assert g == pytest.approx(1e-3)
    assert h == pytest.approx(1e-3 / 0.9)
    assert gaps([_stat("round", 1, [3.0, 1.0], 2)]) == (1.0, 1.0)


@pytest.mark.parametrize("h", [1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-9, 1e-14])
def test_no_tolerance_is_above_the_ceiling(h):
    stats = [_stat("round", 1, [1.0, 1.0 - h * 1.0, 0.0], 1)]
    for eps in (1e-3, 1e-6, 1e-7, 1e-10):
        tol, degenerate = tol32(stats, eps)
        assert tol <= 1e-3
        if eps >= FP32_RESOLUTION:
            assert tol <= TOL_CAP
            assert tol == pytest.approx(min(TOL_BASE + TOL_GAP / gaps(stats)[1], TOL_CAP))
            assert degenerate == (gaps(stats)[1] < DEGENERATE_H)
        else:
            assert not degenerate


def test_rank_allowance_counts_the_values_near_the_threshold():
    eps = 1e-3
    S = np.array([1.0, 0.5, 1e-3 + 5e-7, 1e-3 - 5e-7, 1e-3 - 2e-6, 1e-5])
    allow = rank_allowance([_stat("round", 2, S, 3), _stat("zip_lr", 1, S, 3)], eps, 4)
    assert allow == [0, 0, 4, 0, 0]  # 2 + the two values within 1e-6 of 1e-3; zip-up cuts are not rank checks
    want = [1, 3, 3, 2, 1]
    assert ranks_ok([1, 3, 7, 2, 1], want, [_stat("round", 2, S, 3)], eps)
    assert not ranks_ok([1, 3, 8, 2, 1], want, [_stat("round", 2, S, 3)], eps)
    assert not ranks_ok([1, 4, 3, 2, 1], want, [_stat("round", 2, S, 3)], eps)
    # below the FP32 resolution only the cap is checked
    assert ranks_ok([1, 9, 9, 9, 1], want, [], 1e-8, chi=9)
    assert not ranks_ok([1, 10, 9, 9, 1], want, [], 1e-8, chi=9)
