"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/qtt.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qtt.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qtt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_01904_b300 import build
    build.build()
    from paper_2609_01904_b300 import qtt
    return qtt


def test_header_declares_the_step_entry_points():
    names = _declared()
    for must in ("qtt_velocity_mps", "qtt_laplacian_mpo", "qtt_inject_source", "qtt_step", "qtt_sample",
                 "qtt_to_dense"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert sorted(lib.EXPORTED) == _declared()


def test_library_is_built_for_sm_103a_only():
    """The build compiles every source for sm_103a and for no other target
    (checked on the build's own flags; the library's device code is not
    inspected)."""
    from paper_2609_01904_b300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("arch" in f or "gencode" in f for f in build.FLAGS)


def _params(lib, **kw):
    base = dict(n=4, order=1, bc=0, prec=0, chi_max=8, eps=1e-10, chi_zip=0, eps_zip=0.0, chi_c=0, eps_c=0.0,
                use_learned_rank=0, dims=0)
    base.update(kw)
    return lib.qtt_params(**base)


@pytest.mark.parametrize("bad", [dict(n=0), dict(n=15), dict(order=7), dict(bc=3), dict(chi_max=0),
                                 dict(eps=-1.0), dict(eps=1.5), dict(prec=9), dict(use_learned_rank=2),
                                 dict(chi_zip=-1), dict(chi_max=1025), dict(chi_c=-1), dict(dims=1),
                                 dict(dims=3, n=10), dict(eps=float("nan"))])
def test_ctx_create_rejects_bad_params_without_a_device(lib, bad):
    p = _params(lib, **bad)
    h = ctypes.c_void_p()
    st = lib._lib.qtt_ctx_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == lib.QTT_EINVAL
    assert h.value is None
    assert lib.qtt_last_error() != ""


def test_null_arguments_are_rejected(lib):
    assert lib._lib.qtt_ctx_create(None, None, None) == lib.QTT_EINVAL
    assert lib._lib.qtt_ctx_sync(None) == lib.QTT_EINVAL
    assert lib._lib.qtt_step(None, None, None, 0.1, None, None, None, 0.0) == lib.QTT_EINVAL
    assert lib._lib.qtt_to_dense(None, None, None) == lib.QTT_EINVAL
    lib._lib.qtt_ctx_destroy(None)
    lib._lib.qtt_mps_destroy(None)
    lib._lib.qtt_mpo_destroy(None)
