"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/lra.h declares, and its host-side argument validation rejects bad
parameters before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2506_03859_gb300 import lra
from paper_2506_03859_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return lra.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lra.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lra_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lra_create", "lra_sketch", "lra_farpca_run", "lra_result", "lra_copy_omega",
                 "lra_last_error", "lra_destroy", "lra_farpca_host"):
        assert must in names


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    for name in lra.EXPORTS:
        assert name in declared_functions(), name


def test_struct_layouts():
    assert ctypes.sizeof(lra.Params) == 56
    assert ctypes.sizeof(lra.Matrix) == 40
    assert ctypes.sizeof(lra.Result) == 96


def test_host_only_calls(lib):
    assert lib.lra_version() == 1
    assert lra.status_string(0) == "LRA_OK"
    assert lra.status_string(-1) == "LRA_ERR_INVALID_ARG"
    assert lra.status_string(2) == "LRA_BREAKDOWN"
    assert lib.lra_last_error(None) == b""
    assert lib.lra_capacity(None) == -1
    lib.lra_destroy(None)


BAD = [
    dict(m=0, n=10), dict(m=10, n=10, b=0), dict(m=10, n=10, b=11), dict(m=100, n=100, b=65),
    dict(P=-1), dict(P=9), dict(kind=6), dict(eps=0.0), dict(eps=float("nan")), dict(k=101),
    dict(k=91, b=30), dict(kind=lra.SPARSE_SIGN, zeta=0), dict(kind=lra.SPARSE_SIGN, zeta=257),
    dict(kind=lra.SPARSE_SIGN, zeta=101, n=100), dict(p=1.0), dict(p=-0.1), dict(max_blocks=-1),
    dict(max_blocks=11, b=10), dict(flags=128),
]


@pytest.mark.parametrize("bad", BAD)
def test_create_rejects_bad_arguments(lib, bad):
    args = dict(m=200, n=100, eps=1e-2, k=0, b=10, P=1, kind=lra.SPARSE_SIGN, zeta=8, p=0.0, seed=1,
                max_blocks=0, flags=0)
    args.update(bad)
    prm = lra.Params(args["eps"], args["k"], args["b"], args["P"], args["kind"], args["zeta"], args["p"],
                     args["seed"], args["max_blocks"], args["flags"])
    ctx = ctypes.c_void_p()
    s = lib.lra_create(ctypes.byref(ctx), args["m"], args["n"], ctypes.byref(prm), None)
    assert s == lra.ERR_INVALID_ARG
    assert not ctx.value
    assert lib.lra_create(None, 10, 10, ctypes.byref(prm), None) == lra.ERR_INVALID_ARG


def test_other_entry_points_reject_null_and_bad_arguments(lib):
    """Host-side validation of the SVD, serving, batched and sizing entry points
    (each returns before any device call)."""
    r = lra.SvdResult()
    assert lib.lra_svd(None, ctypes.byref(r)) == lra.ERR_INVALID_ARG
    assert lib.lra_workspace_bytes(2000, 1000, None) == lra.ERR_INVALID_ARG
    bad = lra.params(eps=0.0, b=16)  # eps = 0 without a fixed rank
    assert lib.lra_workspace_bytes(2000, 1000, ctypes.byref(bad)) == lra.ERR_INVALID_ARG
    srv = ctypes.c_void_p()
    for slots, budget in ((0, 0), (65, 0), (4, -1)):
        sp = lra.ServerParams(budget, slots, 0)
        assert lib.lra_server_create(ctypes.byref(srv), ctypes.byref(sp)) == lra.ERR_INVALID_ARG
        assert not srv.value
    assert lib.lra_server_submit(None, None) == lra.ERR_INVALID_ARG
    assert lib.lra_server_pending(None) < 0
    lib.lra_server_destroy(None)
    assert lib.lra_batch_create(None, None, 0, None, None) == lra.ERR_INVALID_ARG
    assert lib.lra_batch_steps(None) < 0 and lib.lra_batch_device_bytes(None) < 0
    lib.lra_batch_destroy(None)
    assert lib.lra_device_bytes(None) == -1


def _ws(lib, m, n, **kw):
    prm = lra.params(**kw)
    return int(lib.lra_workspace_bytes(m, n, ctypes.byref(prm)))


@pytest.mark.parametrize("m,n", [(2000, 1000), (20001, 10003), (129, 17), (300, 5000)])
def test_workspace_holds_the_two_digit_images(lib, m, n):
    """The device workspace of the tensor-core engine holds A's two digit images
    (7 f16 digits, 14 bytes per element): the row-scaled one in 128-row tiles of
    16-deep stages over m x n, the column-scaled one likewise over n x m.
    Without them (LRA_FLAG_NO_A_DIGITS or the FP64 SIMT engine) exactly those
    bytes are gone."""
    base = dict(eps=1e-2, b=16, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    up = lambda x, t: -(-x // t) * t  # noqa: E731
    images = 14 * (up(m, 128) * up(n, 16) + up(n, 128) * up(m, 16))
    with_images = _ws(lib, m, n, **base)
    assert with_images - _ws(lib, m, n, flags=lra.FLAG_NO_A_DIGITS, **base) == images
    assert _ws(lib, m, n, flags=lra.FLAG_FP64_SIMT, **base) < with_images - images + 1


def test_workspace_grows_with_the_problem(lib):
    base = dict(eps=1e-2, b=16, P=1, kind=lra.SPARSE_SIGN, zeta=8, seed=1)
    w = _ws(lib, 2000, 1000, **base)
    assert 0 < w < _ws(lib, 4000, 1000, **base)
    assert w < _ws(lib, 2000, 2000, **base)
    assert w <= _ws(lib, 2000, 1000, **dict(base, b=32))
