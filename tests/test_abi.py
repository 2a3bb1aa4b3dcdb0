"""The C-ABI library loads and exports every function include/fof.h declares.

These run without a GPU: only host-side entry points are called (argument
validation, workspace sizing, error strings).
"""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fof.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fof_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_11468_gb300 import build, fof
    build.build()
    return fof.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fof_create", "fof_link", "fof_groups", "fof_destroy", "fof_batch_create",
                 "fof_workspace_bytes", "fof_run_host", "fof_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2003_11468_gb300 import fof
    out = subprocess.run(["nm", "-D", "--defined-only", fof.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(fof_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_strerror_and_argument_errors(lib):
    from paper_2003_11468_gb300 import fof
    assert fof.strerror(0) == "ok"
    for code in range(1, 10):
        assert fof.strerror(code) != "unknown error"
    h = ctypes.c_void_p()
    # invalid geometry is rejected before any device call
    bad = [(0.0, 0.1, 10), (-1.0, 0.1, 10), (1.0, 0.0, 10), (1.0, 0.5, 10), (1.0, 0.6, 10),
           (float("nan"), 0.1, 10), (1.0, float("inf"), 10), (1.0, 0.1, -1), (1.0, 0.1, 2 ** 31)]
    for box, l_x, n in bad:
        assert lib.fof_create(box, l_x, n, ctypes.byref(h)) == fof.FOF_ERR_ARG, (box, l_x, n)
        assert lib.fof_workspace_bytes(box, l_x, n, None) == 0
    assert lib.fof_create(1.0, 0.1, 10, None) == fof.FOF_ERR_ARG
    assert lib.fof_link(None, None, None) == fof.FOF_ERR_ARG
    assert lib.fof_result(None, None, None, None) == fof.FOF_ERR_ARG


def test_workspace_sizing(lib):
    from paper_2003_11468_gb300 import fof
    w1 = fof.fof_workspace_bytes(1.0, 0.00625, 32768)
    w2 = fof.fof_workspace_bytes(1.0, 0.00625, 2 * 32768)
    assert 44 * 32768 < w1 < 200 * 32768
    assert w2 > w1
    wb = fof.fof_batch_workspace_bytes([1.0, 1.0], [0.00625, 0.00625], [32768, 32768])
    # a batch holds both boxes' particle and cell arrays; only the fixed
    # part (status, scan scratch) is shared
    assert 2 * w1 - 8192 <= wb <= 2 * w1
    # cells per axis beyond the limit set by l_x is an argument error
    opt = fof.fof_options()
    opt.cells_per_axis = 1000
    assert fof.fof_workspace_bytes(1.0, 0.00625, 32768, opt) == 0
    opt.cells_per_axis = 100
    assert fof.fof_workspace_bytes(1.0, 0.00625, 32768, opt) > 0
    opt.brick_cells = 3
    assert fof.fof_workspace_bytes(1.0, 0.00625, 32768, opt) == 0


def test_brick_count_limit(lib):
    """Brick indices are matched and scanned as int32: a plan whose boxes
    hold more than 2^31 - 2 bricks in total is an argument error."""
    from paper_2003_11468_gb300 import fof
    opt = fof.fof_options()
    opt.cells_per_axis = 1024
    opt.brick_cells = 1                     # one cell per brick: 1024^3 bricks per box
    assert fof.fof_batch_workspace_bytes([1.0], [1e-4], [10], opt) > 0
    assert fof.fof_batch_workspace_bytes([1.0, 1.0], [1e-4, 1e-4], [10, 10], opt) == 0
