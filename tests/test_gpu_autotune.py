"""The autotuner (qtt_autotune): it measures the candidate launch shapes of
a step's contractions and QR factorisations on the context's own states,
keeps the fastest, and caches the choices in a JSON file.

Checks: the states it is given are left bit for bit unchanged; the cache it
writes is valid JSON naming every tuned bucket with a choice among the
candidates; a second context loads the same choices from the cache; and a
tuned step gives the untuned step's result (the GEMM tile shapes do not
change any sum's order; the QR's threads per CTA change only the order of
its reductions, within FP64 rounding)."""
import json

import numpy as np
import pytest

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


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _dense(q, psi, N):
    import torch
    out = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    q.qtt_to_dense(psi, out)
    q.qtt_ctx_sync(psi.ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
def test_autotune_caches_valid_choices_and_keeps_results(q, tmp_path, prec):
    n, chi, eps = 7, 64, 1e-8
    N = 1 << n
    c = W.layered_model(n, 20.0, 5)
    lam2 = (0.5 / c.max()) ** 2
    prev_h = O.tt_round(W.random_tt_cores(2 * n, chi, 1, decay=0.05), 1e-14, chi)
    cur_h = O.tt_round(W.random_tt_cores(2 * n, chi, 2, decay=0.05), 1e-14, chi)
    path = str(tmp_path / f"tune_{prec}.json")

    def setup():
        ctx = q.qtt_ctx_create(n=n, chi_max=chi, eps=eps, chi_c=16, eps_c=1e-8, prec=prec)
        L = q.qtt_laplacian_mpo(ctx)
        C = q.qtt_velocity_mps(ctx, _t(c))
        return ctx, L, C, q.qtt_mps_from_cores(ctx, prev_h), q.qtt_mps_from_cores(ctx, cur_h)

    ctx, L, C, prev, cur = setup()
    nb = q.qtt_autotune(L, C, lam2, prev, cur, path, reps=2)
    assert nb > 0
    for a, b in zip(q.qtt_mps_get_cores(cur), cur_h):
        assert np.array_equal(a, b)
    doc = json.load(open(path))
    assert len(doc["entries"]) == nb
    for e in doc["entries"]:
        cands = [256, 1024] if e["op"] == 1 else ([16, 32] if e["kind"] <= 1 else [64, 128, 256])
        assert e["choice"] in cands, e
        assert str(e["choice"]) in e["us_per_launch"]
    text = open(path).read()
    # a second context of the same device, form and shape loads the cache
    ctx2, L2, C2, prev2, cur2 = setup()
    assert q.qtt_autotune(L2, C2, lam2, prev2, cur2, path, reps=2) == nb
    assert open(path).read() == text
    q.qtt_step(L2, C2, lam2, prev2, cur2, (N // 2, 3), 0.2)
    # reference: the same step on a context with the built-in choices
    ctx3, L3, C3, prev3, cur3 = setup()
    q.qtt_step(L3, C3, lam2, prev3, cur3, (N // 2, 3), 0.2)
    a, b = _dense(q, cur2, N), _dense(q, cur3, N)
    tol = 1e-12 if prec == "fp64" else 1e-4
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol
