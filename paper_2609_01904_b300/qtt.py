"""ctypes binding of the C ABI in include/qtt.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device buffers are torch CUDA tensors (float64 /
int64, contiguous) passed by pointer, handles are opaque wrappers.  A missing
or unloadable ``libqtt.so`` raises at import; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqtt.so")

QTT_OK, QTT_EINVAL, QTT_ENOMEM, QTT_ECUDA, QTT_ENOCONV, QTT_ETIMEOUT, QTT_ENONFINITE = range(7)
ORDERS = {"sequential": 0, "interleaved": 1}
BCS = {"periodic": 0, "zero": 1}
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16": 2, "fp32": 3, "tf32x3": 4}
STATUS_NAMES = {0: "QTT_OK", 1: "QTT_EINVAL", 2: "QTT_ENOMEM", 3: "QTT_ECUDA", 4: "QTT_ENOCONV",
                5: "QTT_ETIMEOUT", 6: "QTT_ENONFINITE"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_01904_b300.build`")
_lib = ctypes.CDLL(LIB_PATH)


class qtt_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("order", ctypes.c_int), ("bc", ctypes.c_int), ("prec", ctypes.c_int),
                ("chi_max", ctypes.c_int), ("eps", ctypes.c_double), ("chi_zip", ctypes.c_int),
                ("eps_zip", ctypes.c_double), ("chi_c", ctypes.c_int), ("eps_c", ctypes.c_double),
                ("use_learned_rank", ctypes.c_int), ("dims", ctypes.c_int)]


class QttError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.qtt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_D = ctypes.c_double
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_PL = ctypes.POINTER(ctypes.c_long)

QTT_KCLASSES = 11
KERNEL_CLASSES = ["gemm", "qr", "jacobi", "svd_post", "mpo_apply", "mps_sum", "copy", "fdtd", "refine", "other",
                  "pivot"]


class qtt_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_long * QTT_KCLASSES), ("ms", ctypes.c_double * QTT_KCLASSES),
                ("svd_logged", ctypes.c_long), ("svd_flops", ctypes.c_double), ("svd_sweeps", ctypes.c_long),
                ("flops", ctypes.c_double * QTT_KCLASSES)]


_SIGS = {
    "qtt_ctx_create": [ctypes.POINTER(qtt_params), _P, ctypes.POINTER(_P)],
    "qtt_ctx_sync": [_P],
    "qtt_mps_create_zero": [_P, ctypes.POINTER(_P)],
    "qtt_mps_from_dense": [_P, _P, _I, ctypes.POINTER(_P)],
    "qtt_mps_from_cores": [_P, _PI, _PD, ctypes.POINTER(_P)],
    "qtt_mps_get_cores": [_P, _P, _PI, _PD, _L],
    "qtt_mps_ranks": [_P, _P, _PI],
    "qtt_velocity_mps": [_P, _P, _I, ctypes.POINTER(_P)],
    "qtt_laplacian_mpo": [_P, ctypes.POINTER(_P)],
    "qtt_mpo_bonds": [_P, _PI],
    "qtt_inject_source": [_P, _P, _L, _L, _D],
    "qtt_step": [_P, _P, _P, _D, _P, _P, _PL, _D],
    "qtt_sample": [_P, _P, _P, _P, _L, _P],
    "qtt_to_dense": [_P, _P, _P],
    "qtt_svd_trunc": [_P, _P, _I, _I, _D, _I, _P, _P, _P, _PI],
    "qtt_svd_trunc_noalloc": [_P, _I, _I, _D, _I, _P, _P, _P, _PI, _P],
    "qtt_fdtd_step": [_P, _P, _D, _P, _P, _P, _L, _L, _D],
    "qtt_last_step_discarded": [_P, _PD],
    "qtt_profile_start": [_P, _I, _I],
    "qtt_batch_create": [ctypes.POINTER(qtt_params), _I, _PI, _P, ctypes.POINTER(_P)],
    "qtt_step_batched": [_P, _P, _P, _D, ctypes.POINTER(_P), ctypes.POINTER(_P), _PL, _PD],
    "qtt_profile_read": [_P, ctypes.POINTER(qtt_profile)],
    "qtt_step_graph": [_P, _P, _P, _D, _P, _P, _PL, _D],
    "qtt_batch_set_graphs": [_P, _I],
    "qtt_mps_save": [_P, _P, ctypes.c_char_p],
    "qtt_mps_load": [_P, ctypes.c_char_p, ctypes.POINTER(_P)],
    "qtt_mlp_create": [ctypes.POINTER(ctypes.c_float), _I, _P, ctypes.POINTER(_P)],
    "qtt_mlp_forward": [_P, _P, _I, _P],
    "qtt_mlp_grad": [_P, _P, _P, _I, _P, _P],
    "qtt_mlp_adam_step": [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float],
    "qtt_mlp_get_params": [_P, ctypes.POINTER(ctypes.c_float)],
    "qtt_rank_features": [_P, _I, _P, _P, _I, _D, _I, _I, _P, _P],
    "qtt_step_features": [_P, _P, _P],
    "qtt_set_rank_model": [_P, _P, _P, _I, _I, _I],
    "qtt_set_proposals": [_P, _PI],
    "qtt_get_proposals": [_P, _PI],
    "qtt_learned_stats": [_P, _PL, _PL],
    "qtt_set_limits": [_P, _D, _I],
    "qtt_gemm": [_P, _I, _I, _I, _I, _I, _I, _P, _I, _P, _I, _P, _I, _D, _D, _I],
    "qtt_autotune": [_P, _P, _P, _D, _P, _P, ctypes.c_char_p, _I, _PI],
    "qtt_a_operator_mpo": [_P, _P, _P, _D, ctypes.POINTER(_P)],
    "qtt_step_fused": [_P, _P, _P, _P, _PL, _D],
    "qtt_inject_source_3d": [_P, _P, _L, _L, _L, _D],
    "qtt_sample_3d": [_P, _P, _P, _P, _P, _L, _P],
    "qtt_fdtd_step_3d": [_P, _P, _D, _P, _P, _P, _L, _L, _L, _D],
    "qtt_peak_probe": [_I, _PD, _P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
for _name in ("qtt_ctx_destroy", "qtt_mps_destroy", "qtt_mpo_destroy", "qtt_batch_destroy", "qtt_mlp_destroy"):
    getattr(_lib, _name).argtypes = [_P]
    getattr(_lib, _name).restype = None
_lib.qtt_batch_ctx.argtypes = [_P, _I]
_lib.qtt_batch_ctx.restype = _P
_lib.qtt_mlp_param_count.argtypes = []
_lib.qtt_mlp_param_count.restype = _I
_lib.qtt_last_error.argtypes = []
_lib.qtt_last_error.restype = ctypes.c_char_p

# every symbol include/qtt.h declares
EXPORTED = sorted(list(_SIGS) + ["qtt_ctx_destroy", "qtt_mps_destroy", "qtt_mpo_destroy", "qtt_last_error",
                                  "qtt_batch_destroy", "qtt_batch_ctx", "qtt_mlp_destroy", "qtt_mlp_param_count"])


def _check(st: int, where: str) -> None:
    if st != QTT_OK:
        raise QttError(st, where)


def _dev_ptr(t, dtype_name: str = "float64") -> int:
    import torch
    want = {"float64": torch.float64, "int64": torch.int64, "float32": torch.float32,
            "int32": torch.int32}[dtype_name]
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != want or not t.is_contiguous():
        raise TypeError(f"expected a contiguous CUDA {dtype_name} tensor")
    return t.data_ptr()


def _ptr(t) -> _P:
    """Device pointer of a contiguous CUDA tensor of any of the accepted types."""
    import torch
    names = {torch.float64: "float64", torch.float32: "float32", torch.int32: "int32", torch.int64: "int64"}
    if not isinstance(t, torch.Tensor) or t.dtype not in names:
        raise TypeError("expected a CUDA tensor of float64, float32, int32 or int64")
    return _P(_dev_ptr(t, names[t.dtype]))


class Ctx:
    def __init__(self, handle: int, params: qtt_params, owner=None):
        self.h = handle
        self.params = params
        self.owner = owner  # a batch owns its shots' contexts; states keep it alive

    @property
    def n(self) -> int:
        return self.params.n

    @property
    def dims(self) -> int:
        return 3 if self.params.dims == 3 else 2

    @property
    def d(self) -> int:
        return self.dims * self.params.n

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "owner", None) is None:
            _lib.qtt_ctx_destroy(self.h)
        self.h = None


class Mps:
    def __init__(self, handle: int, ctx: Ctx):
        self.h = handle
        self.ctx = ctx

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qtt_mps_destroy(self.h)
            self.h = None


class Mpo:
    def __init__(self, handle: int, ctx: Ctx):
        self.h = handle
        self.ctx = ctx

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qtt_mpo_destroy(self.h)
            self.h = None


def qtt_last_error() -> str:
    return _lib.qtt_last_error().decode(errors="replace")


def qtt_ctx_create(n: int, order: str = "interleaved", bc: str = "periodic", chi_max: int = 32,
                   eps: float = 1e-10, chi_zip: int = 0, eps_zip: float = 0.0, chi_c: int = 0,
                   eps_c: float = 0.0, prec: str = "fp64", stream=None, learned: bool = False, dims: int = 2) -> Ctx:
    """Context on the current CUDA device; ``stream`` is a torch.cuda.Stream
    (default: torch's current stream); dims = 3 for the 3D extension."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    p = qtt_params(n, ORDERS[order], BCS[bc], PRECISIONS[prec], chi_max, eps, chi_zip, eps_zip, chi_c, eps_c,
                   int(learned), int(dims))
    h = _P()
    _check(_lib.qtt_ctx_create(ctypes.byref(p), _P(stream.cuda_stream), ctypes.byref(h)), "qtt_ctx_create")
    return Ctx(h.value, p)


def qtt_ctx_destroy(ctx: Ctx) -> None:
    if ctx.h:
        _lib.qtt_ctx_destroy(ctx.h)
        ctx.h = None


def qtt_mps_destroy(psi: Mps) -> None:
    if psi.h:
        _lib.qtt_mps_destroy(psi.h)
        psi.h = None


def qtt_mpo_destroy(L: Mpo) -> None:
    if L.h:
        _lib.qtt_mpo_destroy(L.h)
        L.h = None


def qtt_ctx_sync(ctx: Ctx) -> None:
    _check(_lib.qtt_ctx_sync(ctx.h), "qtt_ctx_sync")


def qtt_mps_create_zero(ctx: Ctx) -> Mps:
    h = _P()
    _check(_lib.qtt_mps_create_zero(ctx.h, ctypes.byref(h)), "qtt_mps_create_zero")
    return Mps(h.value, ctx)


def qtt_mps_from_dense(ctx: Ctx, grid) -> Mps:
    """grid: CUDA float64 tensor (N, N) or a host numpy array."""
    h = _P()
    ptr, on_dev, keep = _grid_arg(grid)
    _check(_lib.qtt_mps_from_dense(ctx.h, _P(ptr), on_dev, ctypes.byref(h)), "qtt_mps_from_dense")
    del keep
    return Mps(h.value, ctx)


def qtt_velocity_mps(ctx: Ctx, c_grid) -> Mps:
    h = _P()
    ptr, on_dev, keep = _grid_arg(c_grid)
    _check(_lib.qtt_velocity_mps(ctx.h, _P(ptr), on_dev, ctypes.byref(h)), "qtt_velocity_mps")
    del keep
    return Mps(h.value, ctx)


def _grid_arg(g):
    import numpy as np
    if isinstance(g, np.ndarray):
        a = np.ascontiguousarray(g, dtype=np.float64)
        return a.ctypes.data, 0, a
    return _dev_ptr(g), 1, g


def qtt_mps_from_cores(ctx: Ctx, cores) -> Mps:
    """cores: list of d host arrays [r_k][2][r_{k+1}]."""
    import numpy as np
    ranks = [1] + [int(c.shape[2]) for c in cores]
    flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in cores]))
    r = (ctypes.c_int * len(ranks))(*ranks)
    h = _P()
    _check(_lib.qtt_mps_from_cores(ctx.h, r, flat.ctypes.data_as(_PD), ctypes.byref(h)), "qtt_mps_from_cores")
    return Mps(h.value, ctx)


def qtt_mps_ranks(psi: Mps) -> list[int]:
    r = (ctypes.c_int * (psi.ctx.d + 1))()
    _check(_lib.qtt_mps_ranks(psi.ctx.h, psi.h, r), "qtt_mps_ranks")
    return list(r)


def qtt_mps_get_cores(psi: Mps):
    """Host copy of the cores as a list of numpy arrays."""
    import numpy as np
    ranks = qtt_mps_ranks(psi)
    d = psi.ctx.d
    tot = sum(ranks[k] * 2 * ranks[k + 1] for k in range(d))
    buf = np.empty(max(tot, 1), dtype=np.float64)
    r = (ctypes.c_int * (d + 1))()
    _check(_lib.qtt_mps_get_cores(psi.ctx.h, psi.h, r, buf.ctypes.data_as(_PD), tot), "qtt_mps_get_cores")
    out, o = [], 0
    for k in range(d):
        sz = ranks[k] * 2 * ranks[k + 1]
        out.append(buf[o:o + sz].reshape(ranks[k], 2, ranks[k + 1]).copy())
        o += sz
    return out


def qtt_laplacian_mpo(ctx: Ctx) -> Mpo:
    h = _P()
    _check(_lib.qtt_laplacian_mpo(ctx.h, ctypes.byref(h)), "qtt_laplacian_mpo")
    return Mpo(h.value, ctx)


def qtt_mpo_bonds(L: Mpo) -> list[int]:
    b = (ctypes.c_int * (L.ctx.d + 1))()
    _check(_lib.qtt_mpo_bonds(L.h, b), "qtt_mpo_bonds")
    return list(b)


def _src(src):
    """A grid point (2 or 3 coordinates) as the C array the step calls take."""
    if src is None:
        return None
    return (ctypes.c_long * len(src))(*[int(v) for v in src])


def qtt_inject_source_3d(psi: Mps, ix: int, iy: int, iz: int, amp: float) -> None:
    _check(_lib.qtt_inject_source_3d(psi.ctx.h, psi.h, ix, iy, iz, amp), "qtt_inject_source_3d")


def qtt_sample_3d(psi: Mps, ix, iy, iz, out) -> None:
    """ix, iy, iz: CUDA int64 tensors; out: CUDA float64 tensor of the same length."""
    n = ix.numel()
    _check(_lib.qtt_sample_3d(psi.ctx.h, psi.h, _P(_dev_ptr(ix, "int64")), _P(_dev_ptr(iy, "int64")),
                              _P(_dev_ptr(iz, "int64")), n, _P(_dev_ptr(out))), "qtt_sample_3d")


def qtt_fdtd_step_3d(ctx: Ctx, c2, lambda2: float, u_prev, u_cur, u_next, src=None, amp: float = 0.0) -> None:
    sx, sy, sz = (-1, -1, -1) if src is None else (int(src[0]), int(src[1]), int(src[2]))
    _check(_lib.qtt_fdtd_step_3d(ctx.h, _P(_dev_ptr(c2)), lambda2, _P(_dev_ptr(u_prev)), _P(_dev_ptr(u_cur)),
                                 _P(_dev_ptr(u_next)), sx, sy, sz, amp), "qtt_fdtd_step_3d")


def qtt_inject_source(psi: Mps, ix: int, iz: int, amp: float) -> None:
    _check(_lib.qtt_inject_source(psi.ctx.h, psi.h, ix, iz, amp), "qtt_inject_source")


def qtt_step_graph(L: Mpo, c2: Mps, lambda2: float, psi_prev: Mps, psi_cur: Mps, src=None, amp: float = 0.0) -> None:
    """qtt_step replayed from a CUDA graph captured on the first call."""
    s = _src(src)
    _check(_lib.qtt_step_graph(psi_cur.ctx.h, L.h, c2.h, lambda2, psi_prev.h, psi_cur.h, s, amp), "qtt_step_graph")


def qtt_a_operator_mpo(L: Mpo, c2: Mps, lambda2: float) -> Mpo:
    """MPO of the Eq. 7 transition operator 2I + lambda^2 C^2 L."""
    h = _P()
    _check(_lib.qtt_a_operator_mpo(c2.ctx.h, L.h, c2.h, lambda2, ctypes.byref(h)), "qtt_a_operator_mpo")
    return Mpo(h.value, c2.ctx)


def qtt_step_fused(A: Mpo, psi_prev: Mps, psi_cur: Mps, src=None, amp: float = 0.0) -> None:
    """Eq. 7 with A applied in one zip-up; handles rotate as in qtt_step."""
    s = _src(src)
    _check(_lib.qtt_step_fused(psi_cur.ctx.h, A.h, psi_prev.h, psi_cur.h, s, amp), "qtt_step_fused")


def qtt_step(L: Mpo, c2: Mps, lambda2: float, psi_prev: Mps, psi_cur: Mps, src=None, amp: float = 0.0) -> None:
    """Eq. 17: on return psi_prev holds u^k and psi_cur holds u^{k+1}."""
    s = _src(src)
    _check(_lib.qtt_step(psi_cur.ctx.h, L.h, c2.h, lambda2, psi_prev.h, psi_cur.h, s, amp), "qtt_step")


def qtt_sample(psi: Mps, ix, iz, out) -> None:
    """ix, iz: CUDA int64 tensors; out: CUDA float64 tensor of the same length."""
    n = ix.numel()
    _check(_lib.qtt_sample(psi.ctx.h, psi.h, _P(_dev_ptr(ix, "int64")), _P(_dev_ptr(iz, "int64")), n,
                           _P(_dev_ptr(out))), "qtt_sample")


def qtt_to_dense(psi: Mps, out) -> None:
    """out: CUDA float64 tensor (N, N)."""
    _check(_lib.qtt_to_dense(psi.ctx.h, psi.h, _P(_dev_ptr(out))), "qtt_to_dense")


def qtt_svd_trunc(ctx: Ctx, M, eps: float, chi: int = 0):
    """Truncated SVD of a CUDA float64 matrix (m, n): returns (U, S, Vt, r)."""
    import torch
    m, n = M.shape
    k = min(m, n)
    U = torch.zeros((m, k), dtype=torch.float64, device=M.device)
    S = torch.zeros((k,), dtype=torch.float64, device=M.device)
    Vt = torch.zeros((k, n), dtype=torch.float64, device=M.device)
    r = ctypes.c_int(0)
    _check(_lib.qtt_svd_trunc(ctx.h, _P(_dev_ptr(M)), m, n, eps, chi, _P(U.data_ptr()), _P(S.data_ptr()),
                              _P(Vt.data_ptr()), ctypes.byref(r)), "qtt_svd_trunc")
    r = r.value
    return U.view(-1)[: m * r].view(m, r), S[:r], Vt[:r], r


def qtt_svd_trunc_noalloc(M, U, S, Vt, eps: float, chi: int = 0, stream=None) -> int:
    """The no-allocation truncated SVD: every buffer (CUDA float64, shapes
    (m, n), (m, k), (k,), (k, n) with k = min(m, n)) is the caller's.
    Returns the kept rank."""
    import torch
    m, n = M.shape
    if stream is None:
        stream = torch.cuda.current_stream()
    r = ctypes.c_int(0)
    _check(_lib.qtt_svd_trunc_noalloc(_P(_dev_ptr(M)), m, n, eps, chi, _P(_dev_ptr(U)), _P(_dev_ptr(S)),
                                      _P(_dev_ptr(Vt)), ctypes.byref(r), _P(stream.cuda_stream)),
           "qtt_svd_trunc_noalloc")
    return r.value


def qtt_fdtd_step(ctx: Ctx, c2, lambda2: float, u_prev, u_cur, u_next, src=None, amp: float = 0.0) -> None:
    sx, sz = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    _check(_lib.qtt_fdtd_step(ctx.h, _P(_dev_ptr(c2)), lambda2, _P(_dev_ptr(u_prev)), _P(_dev_ptr(u_cur)),
                              _P(_dev_ptr(u_next)), sx, sz, amp), "qtt_fdtd_step")


def qtt_last_step_discarded(ctx: Ctx):
    import numpy as np
    out = np.zeros(3 * (ctx.d - 1))
    _check(_lib.qtt_last_step_discarded(ctx.h, out.ctypes.data_as(_PD)), "qtt_last_step_discarded")
    return out.reshape(3, ctx.d - 1)


class _BatchHandle:
    def __init__(self, handle: int):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qtt_batch_destroy(self.h)
            self.h = None


class Batch:
    """Handle of a qtt_batch; .ctxs[i] is shot i's context.  The C batch is
    destroyed once the Batch, its contexts and their states are all gone."""

    def __init__(self, hold: _BatchHandle, ctxs: list):
        self.hold = hold
        self.ctxs = ctxs

    @property
    def h(self) -> int:
        return self.hold.h


def qtt_batch_create(n: int, nshots: int, chi_per_shot=None, order: str = "interleaved", bc: str = "periodic",
                     chi_max: int = 32, eps: float = 1e-10, chi_c: int = 0, eps_c: float = 0.0, prec: str = "fp64",
                     stream=None, learned: bool = False) -> Batch:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    p = qtt_params(n, ORDERS[order], BCS[bc], PRECISIONS[prec], chi_max, eps, 0, 0.0, chi_c, eps_c, int(learned), 2)
    chis = None
    if chi_per_shot is not None:
        chis = (ctypes.c_int * nshots)(*[int(x) for x in chi_per_shot])
    h = _P()
    _check(_lib.qtt_batch_create(ctypes.byref(p), nshots, chis, _P(stream.cuda_stream), ctypes.byref(h)),
           "qtt_batch_create")
    hold = _BatchHandle(h.value)
    ctxs = []
    for i in range(nshots):
        chi_i = int(chi_per_shot[i]) if chi_per_shot is not None and int(chi_per_shot[i]) > 0 else chi_max
        pi = qtt_params(p.n, p.order, p.bc, p.prec, chi_i, eps, 0, 0.0, chi_c, eps_c, int(learned), 2)
        ctxs.append(Ctx(_lib.qtt_batch_ctx(hold.h, i), pi, owner=hold))
    return Batch(hold, ctxs)


def qtt_batch_ctx(batch: Batch, shot: int) -> Ctx:
    return batch.ctxs[shot]


def qtt_batch_destroy(batch: Batch) -> None:
    """Drops the Python references; the C batch goes with the last state."""
    batch.ctxs = []
    batch.hold = None


def qtt_batch_set_graphs(batch: Batch, on: bool = True) -> None:
    _check(_lib.qtt_batch_set_graphs(batch.h, int(on)), "qtt_batch_set_graphs")


def qtt_step_batched(batch: Batch, L: Mpo, c2: Mps, lambda2: float, prev: list, cur: list, src=None,
                     amp=None) -> None:
    n = len(batch.ctxs)
    P = (_P * n)(*[x.h for x in prev])
    C = (_P * n)(*[x.h for x in cur])
    s = a = None
    if src is not None:
        flat = [int(v) for xy in src for v in xy]
        s = (ctypes.c_long * len(flat))(*flat)
        a = (ctypes.c_double * n)(*[float(v) for v in amp])
    _check(_lib.qtt_step_batched(batch.h, L.h, c2.h, lambda2, P, C, s, a), "qtt_step_batched")
    # the library exchanged each pair's buffers; the handles keep their roles


def qtt_mps_save(psi: Mps, path: str) -> None:
    _check(_lib.qtt_mps_save(psi.ctx.h, psi.h, os.fsencode(path)), "qtt_mps_save")


def qtt_mps_load(ctx: Ctx, path: str) -> Mps:
    h = _P()
    _check(_lib.qtt_mps_load(ctx.h, os.fsencode(path), ctypes.byref(h)), "qtt_mps_load")
    return Mps(h.value, ctx)


class Mlp:
    """Handle of a qtt_mlp (the rank-proposal network) and its stream."""

    def __init__(self, handle: int, stream):
        self.h = handle
        self.stream = stream

    def __del__(self):
        if getattr(self, "h", None):
            _lib.qtt_mlp_destroy(self.h)
            self.h = None


def qtt_mlp_param_count() -> int:
    return int(_lib.qtt_mlp_param_count())


def qtt_mlp_create(params, max_batch: int, stream=None) -> Mlp:
    """params: host float32 array of qtt_mlp_param_count() values."""
    import numpy as np
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != qtt_mlp_param_count():
        raise ValueError("wrong parameter count")
    h = _P()
    _check(_lib.qtt_mlp_create(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(max_batch),
                               _P(stream.cuda_stream), ctypes.byref(h)), "qtt_mlp_create")
    return Mlp(h.value, stream)


def qtt_mlp_destroy(m: Mlp) -> None:
    m.__del__()


def qtt_mlp_forward(m: Mlp, X, y) -> None:
    """X: float32 CUDA tensor n x 40; y: float32 CUDA tensor n."""
    _check(_lib.qtt_mlp_forward(m.h, _ptr(X), int(X.shape[0]), _ptr(y)), "qtt_mlp_forward")


def qtt_mlp_grad(m: Mlp, X, t, loss=None, grad=None) -> None:
    _check(_lib.qtt_mlp_grad(m.h, _ptr(X), _ptr(t), int(X.shape[0]), _ptr(loss) if loss is not None else None,
                             _ptr(grad) if grad is not None else None), "qtt_mlp_grad")


def qtt_mlp_adam_step(m: Mlp, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    _check(_lib.qtt_mlp_adam_step(m.h, lr, beta1, beta2, eps), "qtt_mlp_adam_step")


def qtt_mlp_get_params(m: Mlp):
    import numpy as np
    out = np.empty(qtt_mlp_param_count(), dtype=np.float32)
    _check(_lib.qtt_mlp_get_params(m.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "qtt_mlp_get_params")
    return out


def qtt_rank_features(S, lens, ranks, nb: int, eps: float, chi: int, d: int, X, stream=None) -> None:
    """S: float64 CUDA tensor (rows x lds); lens, ranks: int32 CUDA tensors;
    X: float32 CUDA tensor nb x 40."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.qtt_rank_features(_ptr(S), int(S.shape[1]), _ptr(lens), _ptr(ranks), nb, eps, chi, d, _ptr(X),
                                  _P(stream.cuda_stream)), "qtt_rank_features")


def qtt_step_features(psi: Mps, X) -> None:
    _check(_lib.qtt_step_features(psi.ctx.h, psi.h, _ptr(X)), "qtt_step_features")


def qtt_set_rank_model(ctx: Ctx, mlp, sketch, oversample: int = 16) -> None:
    """mlp: Mlp or None; sketch: float64 CUDA tensor rows x cols (kept alive
    by the caller) or None to turn the learned rounding off."""
    ctx._sketch = sketch
    ctx._mlp = mlp
    if sketch is None:
        _check(_lib.qtt_set_rank_model(ctx.h, None, None, 0, 0, 0), "qtt_set_rank_model")
        return
    _check(_lib.qtt_set_rank_model(ctx.h, mlp.h if mlp is not None else None, _ptr(sketch), int(sketch.shape[0]),
                                   int(sketch.shape[1]), int(oversample)), "qtt_set_rank_model")


def qtt_set_proposals(ctx: Ctx, prop) -> None:
    a = (ctypes.c_int * (ctx.d + 1))(*[int(x) for x in prop])
    _check(_lib.qtt_set_proposals(ctx.h, a), "qtt_set_proposals")


def qtt_get_proposals(ctx: Ctx) -> list:
    a = (ctypes.c_int * (ctx.d + 1))()
    _check(_lib.qtt_get_proposals(ctx.h, a), "qtt_get_proposals")
    return list(a)


def qtt_learned_stats(ctx: Ctx) -> tuple:
    a, b = ctypes.c_long(), ctypes.c_long()
    _check(_lib.qtt_learned_stats(ctx.h, ctypes.byref(a), ctypes.byref(b)), "qtt_learned_stats")
    return a.value, b.value


def qtt_profile_start(ctx: Ctx, timing: bool = False, log_svd: bool = False) -> None:
    _check(_lib.qtt_profile_start(ctx.h, int(timing), int(log_svd)), "qtt_profile_start")


def qtt_profile_read(ctx: Ctx) -> dict:
    p = qtt_profile()
    _check(_lib.qtt_profile_read(ctx.h, ctypes.byref(p)), "qtt_profile_read")
    return {"launches": dict(zip(KERNEL_CLASSES, list(p.launches))), "ms": dict(zip(KERNEL_CLASSES, list(p.ms))),
            "svd_logged": p.svd_logged, "svd_flops": p.svd_flops, "svd_sweeps": p.svd_sweeps,
            "flops": dict(zip(KERNEL_CLASSES, list(p.flops)))}


GEMM_KINDS = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16": 4}


def qtt_gemm(ctx: Ctx, kind: str, A, B, C, alpha: float = 1.0, beta: float = 0.0, a_trans: bool = False,
             b_trans: bool = False, tile_n: int = 0) -> None:
    """C = alpha op(A) op(B) + beta C on CUDA float64 tensors (row-major 2-D;
    op transposes a stored matrix when *_trans)."""
    m, k = (A.shape[1], A.shape[0]) if a_trans else (A.shape[0], A.shape[1])
    n = B.shape[0] if b_trans else B.shape[1]
    _check(_lib.qtt_gemm(ctx.h, GEMM_KINDS[kind], int(a_trans), int(b_trans), m, n, k, _P(_dev_ptr(A)),
                         A.stride(0), _P(_dev_ptr(B)), B.stride(0), _P(_dev_ptr(C)), C.stride(0), alpha, beta,
                         int(tile_n)), "qtt_gemm")


def qtt_autotune(L: Mpo, c2: Mps, lambda2: float, psi_prev: Mps, psi_cur: Mps, cache_path: str | None = None,
                 reps: int = 5) -> int:
    """Autotune the launch shapes of the step on the states' context (see
    include/qtt.h); returns the number of buckets tuned."""
    n = ctypes.c_int(0)
    _check(_lib.qtt_autotune(psi_cur.ctx.h, L.h, c2.h, lambda2, psi_prev.h, psi_cur.h,
                             os.fsencode(cache_path) if cache_path else None, int(reps), ctypes.byref(n)),
           "qtt_autotune")
    return n.value


def qtt_set_limits(ctx: Ctx, wait_limit_s: float = 0.0, max_sweeps: int = 0) -> None:
    """Bounded-wait limit (seconds) and FP64 Jacobi sweep limit; 0 = defaults."""
    _check(_lib.qtt_set_limits(ctx.h, float(wait_limit_s), int(max_sweeps)), "qtt_set_limits")


def qtt_peak_probe(kind: str, stream=None) -> float:
    """Measured FMA peak of the device in TFLOP/s: kind "fp32" or "fp64"."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    _check(_lib.qtt_peak_probe({"fp32": 0, "fp64": 1}[kind], ctypes.byref(out), _P(stream.cuda_stream)),
           "qtt_peak_probe")
    return out.value


__all__ = [n for n in EXPORTED] + ["Ctx", "Mps", "Mpo", "QttError", "qtt_params", "EXPORTED", "LIB_PATH"]
