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
