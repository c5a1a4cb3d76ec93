"""The core-contraction kernel (qtt_gemm) in every operand form, against
numpy's FP64 product of the same FP64 inputs.

Tolerance: the standard bound of a rounded dot product, elementwise,
    |C - C_ref|_ij <= gamma * (|op(A)| |op(B)|)_ij,
gamma = 2 u_in + K u_acc (+ FP64 rounding of the alpha / beta epilogue), with u_in the unit roundoff of
the operand type (the inputs are rounded to it: FP64 2^-53, FP32 2^-24,
TF32 2^-11, BF16 2^-8; 3xTF32 keeps x - hi to TF32, so its operands carry
2^-22 and the dropped lo*lo product another 2^-22) and u_acc that of the
accumulator (FP64 2^-53, else FP32 2^-24).  Shapes span several 128-row and
N tiles with ragged tails and K chunks that are not multiples of the chunk
(32 TF32 / 64 BF16 values); both storage orders of both operands (the two
load paths of the kernel), alpha / beta, K = 0 and 1 x 1."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U_IN = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "tf32x3": 3 * 2.0 ** -22, "bf16": 2.0 ** -8}
U_ACC = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -24, "tf32x3": 2.0 ** -24, "bf16": 2.0 ** -24}


@pytest.fixture(scope="module")
def q():
    import torch  # noqa: F401
    from paper_2609_01904_b300 import build
    build.build()
    from paper_2609_01904_b300 import qtt
    return qtt


@pytest.fixture(scope="module")
def ctx(q):
    return q.qtt_ctx_create(n=6, chi_max=32)


def _run(q, ctx, kind, m, n, k, a_trans, b_trans, alpha, beta, tile_n, seed):
    import torch
    rng = np.random.default_rng(seed)
    Ah = rng.standard_normal((k, m) if a_trans else (m, k)) * np.exp(rng.uniform(-3, 3, (1, 1)))
    Bh = rng.standard_normal((n, k) if b_trans else (k, n))
    Ch = rng.standard_normal((m, n))
    A, B = torch.as_tensor(Ah, device="cuda"), torch.as_tensor(Bh, device="cuda")
    C = torch.as_tensor(Ch.copy(), device="cuda")
    q.qtt_gemm(ctx, kind, A, B, C, alpha, beta, a_trans, b_trans, tile_n)
    q.qtt_ctx_sync(ctx)
    opA = Ah.T if a_trans else Ah
    opB = Bh.T if b_trans else Bh
    ref = alpha * (opA @ opB) + beta * Ch
    gamma = 2 * U_IN[kind] + max(k, 1) * U_ACC[kind] + 4 * 2.0 ** -53
    # the product's bound, plus FP64 rounding of the alpha / beta epilogue
    allowed = gamma * abs(alpha) * (np.abs(opA) @ np.abs(opB)) + 8 * 2.0 ** -53 * (np.abs(beta * Ch) + np.abs(ref))
    err = np.abs(C.cpu().numpy() - ref)
    ratio = float(np.max(err / np.maximum(allowed, 1e-300)))
    return ratio, float(np.max(err))


@pytest.mark.parametrize("kind", ["fp64", "fp32", "tf32", "tf32x3", "bf16"])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 7, 3), (128, 64, 32), (200, 300, 130), (640, 256, 128),
                                   (257, 129, 67)])
@pytest.mark.parametrize("a_trans,b_trans", [(False, False), (True, True), (False, True), (True, False)])
def test_contraction_within_the_rounding_bound_of_its_operand_type(q, ctx, kind, m, n, k, a_trans, b_trans):
    ratio, err = _run(q, ctx, kind, m, n, k, a_trans, b_trans, 1.0, 0.0, 0, m * 1000 + n + k)
    assert ratio <= 1.0, (kind, m, n, k, ratio, err)


@pytest.mark.parametrize("kind", ["tf32", "tf32x3", "bf16"])
@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_every_tensor_core_tile_width(q, ctx, kind, tile_n):
    for m, n, k in ((300, 520, 200), (128, 256, 64), (3, 70, 9)):
        ratio, err = _run(q, ctx, kind, m, n, k, False, False, -0.7, 1.3, tile_n, 7 + tile_n + m)
        assert ratio <= 1.0, (kind, tile_n, m, n, k, ratio, err)


@pytest.mark.parametrize("kind", ["fp64", "fp32", "tf32", "tf32x3", "bf16"])
def test_empty_contraction_scales_c(q, ctx, kind):
    import torch
    A = torch.zeros((4, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    Ch = np.arange(20.0).reshape(4, 5)
    C = torch.as_tensor(Ch.copy(), device="cuda")
    # K = 0: C <- beta C (the leading dimension of an empty A is taken as 1)
    q._check(q._lib.qtt_gemm(ctx.h, q.GEMM_KINDS[kind], 0, 0, 4, 5, 0, q._P(A.data_ptr()), 1, q._P(B.data_ptr()),
                             5, q._P(C.data_ptr()), 5, 1.0, 0.5, 0), "qtt_gemm")
    q.qtt_ctx_sync(ctx)
    assert np.array_equal(C.cpu().numpy(), 0.5 * Ch)


def test_bad_arguments_are_rejected(q, ctx):
    import torch
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(q.QttError) as e:
        q.qtt_gemm(ctx, "tf32", A, A, A, tile_n=96)
    assert e.value.status == q.QTT_EINVAL
