"""Shots that run concurrently on the batch's streams must not change each
other's arithmetic: identical shots stepped together give bit-identical
states, equal to the same step taken alone on one stream.

The step's kernels share no memory across contexts, so any difference is a
race inside a kernel that only shows when other kernels share its SMs (the
dataflow QR once read a column's pivot entry in some warps after thread 0 had
updated it; isolated runs hid that, concurrent shots did not).  The state is
the 512x512 layered section at step 1000 with chi = 128 (ranks at the cap:
the zip-ups and the round take every SVD route, and a different rounding at a
cut changes the kept subspace, so any race shows), FP32 and FP64 forms."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2609_01904_b300 import build
    build.build()
    from paper_2609_01904_b300 import qtt
    return qtt


@pytest.fixture(scope="module")
def start(q):
    import torch
    wl = W.config(3)
    c = wl.velocity()
    lam2 = wl.lambda2(c)
    amps = wl.source_amplitudes(c, 1010)
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=128, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec="fp64")
    c_dev = torch.as_tensor(c, device="cuda")
    c2 = c_dev * c_dev
    N = wl.N
    up = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    uc, un = up.clone(), up.clone()
    for k in range(1000):
        q.qtt_fdtd_step(ctx, c2, lam2, up, uc, un, wl.sources[0], float(amps[k]))
        up, uc, un = uc, un, up
    p0 = q.qtt_mps_get_cores(q.qtt_mps_from_dense(ctx, up))
    c0 = q.qtt_mps_get_cores(q.qtt_mps_from_dense(ctx, uc))
    return wl, c_dev, lam2, amps, p0, c0


def _cores(q, psi):
    q.qtt_ctx_sync(psi.ctx)
    return q.qtt_mps_ranks(psi), np.concatenate([x.ravel() for x in q.qtt_mps_get_cores(psi)])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_identical_concurrent_shots_are_bit_identical_to_the_step_alone(q, start, prec):
    wl, c_dev, lam2, amps, p0, c0 = start
    nb, steps = 8, 2 if prec == "fp32" else 1
    src = wl.sources[0]
    # alone: one context, one stream
    ctx = q.qtt_ctx_create(n=wl.n, order=wl.order, bc=wl.bc, chi_max=128, eps=wl.eps, chi_c=wl.chi_c,
                           eps_c=wl.eps_c, prec=prec)
    C, L = q.qtt_velocity_mps(ctx, c_dev), q.qtt_laplacian_mpo(ctx)
    P, Q = q.qtt_mps_from_cores(ctx, p0), q.qtt_mps_from_cores(ctx, c0)
    for k in range(steps):
        q.qtt_step(L, C, lam2, P, Q, src, float(amps[1000 + k]))
    want_r, want = _cores(q, Q)
    # together: nb identical shots on the batch's streams, launched (no graphs)
    batch = q.qtt_batch_create(wl.n, nb, [128] * nb, order=wl.order, bc=wl.bc, chi_max=128, eps=wl.eps,
                               chi_c=wl.chi_c, eps_c=wl.eps_c, prec=prec)
    q.qtt_batch_set_graphs(batch, False)
    Cb, Lb = q.qtt_velocity_mps(batch.ctxs[0], c_dev), q.qtt_laplacian_mpo(batch.ctxs[0])
    prev = [q.qtt_mps_from_cores(batch.ctxs[s], p0) for s in range(nb)]
    cur = [q.qtt_mps_from_cores(batch.ctxs[s], c0) for s in range(nb)]
    for rep in range(3):
        prev = [q.qtt_mps_from_cores(batch.ctxs[s], p0) for s in range(nb)]
        cur = [q.qtt_mps_from_cores(batch.ctxs[s], c0) for s in range(nb)]
        for k in range(steps):
            q.qtt_step_batched(batch, Lb, Cb, lam2, prev, cur, [src] * nb, [float(amps[1000 + k])] * nb)
        for s in range(nb):
            got_r, got = _cores(q, cur[s])
            assert got_r == want_r, (rep, s)
            assert np.array_equal(got, want), (rep, s, float(np.abs(got - want).max()))
