"""CPU oracle for the Friends-of-Friends group finder -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never loads it, and it never loads the product.

The arithmetic lives in ``fof_oracle.c`` (plain C, single thread, compiled
with ``-ffp-contract=off``); this module compiles it on first use and
wraps it with numpy.  See the header of ``fof_oracle.c`` for what each
function computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fof_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc) if missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int32
            lib.fof_oracle_linked.argtypes = [P, P, f64, f64]
            lib.fof_oracle_linked.restype = ctypes.c_int
            lib.fof_oracle_linked_rule.argtypes = [P, P, f64, f64, ctypes.c_int]
            lib.fof_oracle_linked_rule.restype = ctypes.c_int
            lib.fof_oracle_groups_rule.argtypes = [i64, P, f64, f64, ctypes.c_int, P, P]
            lib.fof_oracle_groups_rule.restype = ctypes.c_int
            lib.fof_oracle_brute_rule.argtypes = [i64, P, f64, f64, ctypes.c_int, P]
            lib.fof_oracle_brute_rule.restype = ctypes.c_int
            lib.fof_oracle_linked_many.argtypes = [i64, P, P, f64, f64, P]
            lib.fof_oracle_linked_many.restype = None
            lib.fof_oracle_groups.argtypes = [i64, P, f64, f64, P, P]
            lib.fof_oracle_groups.restype = ctypes.c_int
            lib.fof_oracle_brute.argtypes = [i64, P, f64, f64, P]
            lib.fof_oracle_brute.restype = ctypes.c_int
            lib.fof_oracle_component.argtypes = [i64, P, f64, f64, i64, P, P, P]
            lib.fof_oracle_component.restype = ctypes.c_int
            lib.fof_oracle_catalogue.argtypes = [i64, P, i32, P, i64]
            lib.fof_oracle_catalogue.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _pos(pos) -> np.ndarray:
    a = np.ascontiguousarray(pos, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        a = a.reshape(-1, 3)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def linked(a, b, box: float, l_x: float, strict: bool = False) -> bool:
    """The exact link predicate for two float32 points (strict: distance < l_x)."""
    pa = np.ascontiguousarray(a, dtype=np.float32).reshape(3)
    pb = np.ascontiguousarray(b, dtype=np.float32).reshape(3)
    if strict:
        return bool(_load().fof_oracle_linked_rule(_ptr(pa), _ptr(pb), float(box), float(l_x), 1))
    return bool(_load().fof_oracle_linked(_ptr(pa), _ptr(pb), float(box), float(l_x)))


def linked_many(a, b, box: float, l_x: float) -> np.ndarray:
    """The predicate for each pair of rows of a and b (float32 [m, 3])."""
    pa, pb = _pos(a), _pos(b)
    out = np.empty(pa.shape[0], dtype=np.uint8)
    _load().fof_oracle_linked_many(pa.shape[0], _ptr(pa), _ptr(pb), float(box), float(l_x), _ptr(out))
    return out.astype(bool)


def groups(pos, box: float, l_x: float, strict: bool = False):
    """(ids, sizes): min-index labels and per-label sizes, int32 arrays of n.
    strict: link only pairs at distance < l_x (the naive listing's tie rule)."""
    p = _pos(pos)
    n = p.shape[0]
    ids = np.empty(n, dtype=np.int32)
    sizes = np.empty(n, dtype=np.int32)
    if strict:
        rc = _load().fof_oracle_groups_rule(n, _ptr(p), float(box), float(l_x), 1, _ptr(ids), _ptr(sizes))
    else:
        rc = _load().fof_oracle_groups(n, _ptr(p), float(box), float(l_x), _ptr(ids), _ptr(sizes))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return ids, sizes


def brute(pos, box: float, l_x: float, strict: bool = False) -> np.ndarray:
    """ids by the O(N^2) pair loop with serial union-find (tiny inputs only)."""
    p = _pos(pos)
    n = p.shape[0]
    ids = np.empty(n, dtype=np.int32)
    if strict:
        _load().fof_oracle_brute_rule(n, _ptr(p), float(box), float(l_x), 1, _ptr(ids))
    else:
        _load().fof_oracle_brute(n, _ptr(p), float(box), float(l_x), _ptr(ids))
    return ids


def component(pos, box: float, l_x: float, start: int):
    """(label, members) of the group holding particle `start`."""
    p = _pos(pos)
    n = p.shape[0]
    members = np.empty(max(n, 1), dtype=np.int32)
    cnt = ctypes.c_int64(0)
    lab = ctypes.c_int64(0)
    rc = _load().fof_oracle_component(n, _ptr(p), float(box), float(l_x), int(start),
                                      _ptr(members), ctypes.byref(cnt), ctypes.byref(lab))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return int(lab.value), np.sort(members[: cnt.value])


def catalogue(sizes, min_size: int) -> np.ndarray:
    """(label, size) rows for sizes >= max(min_size, 1), ascending label."""
    s = np.ascontiguousarray(sizes, dtype=np.int32)
    n = s.shape[0]
    lib = _load()
    cnt = lib.fof_oracle_catalogue(n, _ptr(s), int(min_size), None, 0)
    cat = np.empty((max(cnt, 1), 2), dtype=np.int32)
    lib.fof_oracle_catalogue(n, _ptr(s), int(min_size), _ptr(cat), cnt)
    return cat[:cnt]
