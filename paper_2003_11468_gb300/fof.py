"""ctypes binding of the C ABI in include/fof.h (argument marshalling only).

Every function of the header is exposed under the same name and takes the
same arguments, with torch tensors accepted wherever the C side takes a
pointer (their data_ptr() is passed) and torch streams wherever it takes a
cudaStream_t.  All computation happens in libfof_gb300.so; if that library
is missing this module raises on load, there is no fallback.

`FoF` / `FoFBatch` wrap a handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# FOF_LIBRARY=debug loads the build with every neighbour-candidate slot
# checked (bad slots reported as FOF_ERR_INTERNAL); the default is the
# production build
LIB_PATH = os.path.join(HERE, "libfof_gb300_debug.so" if os.environ.get("FOF_LIBRARY") == "debug"
                        else "libfof_gb300.so")

FOF_OK = 0
FOF_ERR_ARG = 1
FOF_ERR_RANGE = 2
FOF_ERR_CAPACITY = 3
FOF_ERR_STATE = 4
FOF_ERR_OOM = 5
FOF_ERR_CUDA = 6
FOF_ERR_TIMEOUT = 7
FOF_ERR_INTERNAL = 8
FOF_ERR_TOO_LARGE = 9


class fof_options(ctypes.Structure):
    _fields_ = [
        ("cells_per_axis", ctypes.c_int32),
        ("brick_cells", ctypes.c_int32),
        ("occupancy", ctypes.c_double),
        ("dense_min", ctypes.c_int32),
        ("retry_cap", ctypes.c_int32),
        ("team_min", ctypes.c_int32),
        ("tie_rule", ctypes.c_int32),
        ("find_variant", ctypes.c_int32),
        ("size_count", ctypes.c_int32),
        ("link_order", ctypes.c_int32),
        ("debug_flags", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


FOF_TIE_LE, FOF_TIE_LT = 0, 1
FOF_FIND_HALVE_DEEP, FOF_FIND_HALVE_ALL, FOF_FIND_FULL, FOF_FIND_NONE = 0, 1, 2, 3
FOF_SIZE_WARP, FOF_SIZE_HASH = 0, 1
FOF_LINK_MIN, FOF_LINK_RANDOM = 0, 1
FOF_DEBUG_UNION_NO_RETRY = 1
FOF_DEBUG_VARIANT_KERNELS = 2


class fof_geometry(ctypes.Structure):
    _fields_ = [
        ("cells_per_axis", ctypes.c_int32),
        ("brick_cells", ctypes.c_int32),
        ("bricks_per_axis", ctypes.c_int32),
        ("sub_cells", ctypes.c_int32),
        ("fine_per_axis", ctypes.c_int32),
        ("inv_fine", ctypes.c_float),
        ("xmax", ctypes.c_float),
        ("t_lo", ctypes.c_float),
        ("t_hi", ctypes.c_float),
        ("bb_reach2", ctypes.c_float),
    ]


class FoFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


_lib = None
_lock = threading.Lock()


def load():
    """Load libfof_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2003_11468_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P, i32, i64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                ctypes.c_size_t)
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "fof_create": ([f64, f64, i64, PP], ctypes.c_int),
            "fof_create_ex": ([f64, f64, i64, P, P, sz, PP], ctypes.c_int),
            "fof_workspace_bytes": ([f64, f64, i64, P], sz),
            "fof_batch_create": ([i32, P, P, P, P, P, sz, PP], ctypes.c_int),
            "fof_batch_workspace_bytes": ([i32, P, P, P, P], sz),
            "fof_link": ([P, P, P], ctypes.c_int),
            "fof_relink": ([P, P, P, P], ctypes.c_int),
            "fof_groups": ([P, P, P, P, i64, i32, P, P, P], ctypes.c_int),
            "fof_groups_async": ([P, P, P, P, i64, i32, P], ctypes.c_int),
            "fof_result": ([P, P, P, P], ctypes.c_int),
            "fof_run_host": ([P, P, P, P, P, i64, i32, P, P, P], ctypes.c_int),
            "fof_run_host_many": ([P, i32, P, P, P, P, i64, i32, P, P, P], ctypes.c_int),
            "fof_graph_build": ([P, P, P, P, P, i64, i32, P], ctypes.c_int),
            "fof_graph_launch": ([P, P], ctypes.c_int),
            "fof_plan_info": ([P, i32, P, P, P], ctypes.c_int),
            "fof_box_geometry": ([f64, f64, i64, P, P], ctypes.c_int),
            "fof_set_timing": ([P, ctypes.c_int], ctypes.c_int),
            "fof_phase_times": ([P, P, P, P, ctypes.c_int], ctypes.c_int),
            "fof_reset_times": ([P], ctypes.c_int),
            "fof_kernel_launches": ([P], i64),
            "fof_destroy": ([P], None),
            "fof_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "fof_run_noalloc": ([f64, f64, i64, P, P, P, P, i64, i32, P, P, P], ctypes.c_int),
            "fof_merge_links": ([i64, P, P, i64, P, P, i64, P, P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x):
    """Pointer of a torch tensor, a numpy array, an int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() > 0 else None
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(code: int, where: str) -> int:
    if code != FOF_OK:
        raise FoFError(code, where)
    return code


def strerror(code: int) -> str:
    return load().fof_strerror(code).decode()


# ---------------------------------------------------------------------------
# the C ABI, same names
# ---------------------------------------------------------------------------

def fof_create(box: float, l_x: float, n: int) -> int:
    h = ctypes.c_void_p()
    _check(load().fof_create(box, l_x, n, ctypes.byref(h)), "fof_create")
    return h.value


def fof_create_ex(box, l_x, n, opt: fof_options | None = None, workspace=None, workspace_bytes=0):
    h = ctypes.c_void_p()
    _check(load().fof_create_ex(box, l_x, n, ctypes.byref(opt) if opt is not None else None,
                                _ptr(workspace), workspace_bytes, ctypes.byref(h)), "fof_create_ex")
    return h.value


def fof_workspace_bytes(box, l_x, n, opt: fof_options | None = None) -> int:
    return load().fof_workspace_bytes(box, l_x, n, ctypes.byref(opt) if opt is not None else None)


def _arrays(boxes, lxs, ns):
    k = len(boxes)
    B = (ctypes.c_double * k)(*boxes)
    X = (ctypes.c_double * k)(*lxs)
    N = (ctypes.c_int64 * k)(*ns)
    return k, B, X, N


def fof_batch_create(boxes, lxs, ns, opt: fof_options | None = None, workspace=None,
                     workspace_bytes=0) -> int:
    k, B, X, N = _arrays(boxes, lxs, ns)
    h = ctypes.c_void_p()
    _check(load().fof_batch_create(k, B, X, N, ctypes.byref(opt) if opt is not None else None,
                                   _ptr(workspace), workspace_bytes, ctypes.byref(h)),
           "fof_batch_create")
    return h.value


def fof_batch_workspace_bytes(boxes, lxs, ns, opt: fof_options | None = None) -> int:
    k, B, X, N = _arrays(boxes, lxs, ns)
    return load().fof_batch_workspace_bytes(k, B, X, N, ctypes.byref(opt) if opt is not None else None)


def fof_link(h, pos, stream=None) -> int:
    return _check(load().fof_link(h, _ptr(pos), _stream(stream)), "fof_link")


def fof_relink(h, pos, stream=None) -> int:
    """fof_link for moved particles; returns the path taken (0, 1 or 2)."""
    path = ctypes.c_int32(-1)
    _check(load().fof_relink(h, _ptr(pos), ctypes.byref(path), _stream(stream)), "fof_relink")
    return path.value


def fof_groups(h, ids, sizes, catalogue, cat_capacity, min_size, nbox=1, stream=None,
               allow_capacity=False):
    """Returns (code, n_groups[list], n_cat[list])."""
    ng = (ctypes.c_int64 * nbox)()
    nk = (ctypes.c_int64 * nbox)()
    code = load().fof_groups(h, _ptr(ids), _ptr(sizes), _ptr(catalogue), cat_capacity, min_size,
                             ng, nk, _stream(stream))
    if code != FOF_OK and not (allow_capacity and code == FOF_ERR_CAPACITY):
        raise FoFError(code, "fof_groups")
    return code, list(ng), list(nk)


def fof_groups_async(h, ids, sizes, catalogue, cat_capacity, min_size, stream=None) -> int:
    return _check(load().fof_groups_async(h, _ptr(ids), _ptr(sizes), _ptr(catalogue), cat_capacity,
                                          min_size, _stream(stream)), "fof_groups_async")


def fof_result(h, nbox=1, stream=None, allow_capacity=False):
    ng = (ctypes.c_int64 * nbox)()
    nk = (ctypes.c_int64 * nbox)()
    code = load().fof_result(h, ng, nk, _stream(stream))
    if code != FOF_OK and not (allow_capacity and code == FOF_ERR_CAPACITY):
        raise FoFError(code, "fof_result")
    return code, list(ng), list(nk)


def fof_run_host(h, pos_host, ids_host, sizes_host, cat_host, cat_capacity, min_size, nbox=1,
                 stream=None, allow_capacity=False):
    ng = (ctypes.c_int64 * nbox)()
    nk = (ctypes.c_int64 * nbox)()
    code = load().fof_run_host(h, _ptr(pos_host), _ptr(ids_host), _ptr(sizes_host), _ptr(cat_host),
                               cat_capacity, min_size, ng, nk, _stream(stream))
    if code != FOF_OK and not (allow_capacity and code == FOF_ERR_CAPACITY):
        raise FoFError(code, "fof_run_host")
    return code, list(ng), list(nk)


def fof_run_host_many(h, pos_hosts, ids_hosts, sizes_hosts, cat_hosts, cat_capacity, min_size, nbox=1,
                      stream=None, allow_capacity=False):
    """fof_run_host over several inputs with overlapped copies; returns
    (code, n_groups[nsteps][nbox], n_cat[nsteps][nbox])."""
    k = len(pos_hosts)
    VP = ctypes.c_void_p * max(k, 1)
    pp = VP(*[_ptr(x) for x in pos_hosts])
    ip = VP(*[_ptr(x) for x in ids_hosts])
    sp = VP(*[_ptr(x) for x in sizes_hosts])
    cp = VP(*[_ptr(x) for x in cat_hosts]) if cat_hosts is not None else None
    ng = (ctypes.c_int64 * max(k * nbox, 1))()
    nk = (ctypes.c_int64 * max(k * nbox, 1))()
    code = load().fof_run_host_many(h, k, pp, ip, sp, cp, cat_capacity, min_size, ng, nk, _stream(stream))
    if code != FOF_OK and not (allow_capacity and code == FOF_ERR_CAPACITY):
        raise FoFError(code, "fof_run_host_many")
    return (code, [list(ng[i * nbox:(i + 1) * nbox]) for i in range(k)],
            [list(nk[i * nbox:(i + 1) * nbox]) for i in range(k)])


def fof_graph_build(h, pos, ids, sizes, catalogue, cat_capacity, min_size, stream) -> int:
    return _check(load().fof_graph_build(h, _ptr(pos), _ptr(ids), _ptr(sizes), _ptr(catalogue),
                                         cat_capacity, min_size, _stream(stream)), "fof_graph_build")


def fof_graph_launch(h, stream) -> int:
    return _check(load().fof_graph_launch(h, _stream(stream)), "fof_graph_launch")


def fof_box_geometry(box, l_x, n, opt: fof_options | None = None) -> fof_geometry:
    out = fof_geometry()
    _check(load().fof_box_geometry(box, l_x, n, ctypes.byref(opt) if opt is not None else None,
                                   ctypes.byref(out)), "fof_box_geometry")
    return out


def fof_plan_info(h, b=0):
    nc, r, nb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().fof_plan_info(h, b, ctypes.byref(nc), ctypes.byref(r), ctypes.byref(nb)),
           "fof_plan_info")
    return nc.value, r.value, nb.value


def fof_set_timing(h, enable: bool) -> int:
    return _check(load().fof_set_timing(h, 1 if enable else 0), "fof_set_timing")


def fof_phase_times(h) -> dict:
    """{phase name: (milliseconds, launches)} summed since the last reset."""
    m = 16
    ms = (ctypes.c_double * m)()
    ln = (ctypes.c_int64 * m)()
    names = (ctypes.c_char_p * m)()
    k = load().fof_phase_times(h, ms, ln, names, m)
    if k < 0:
        raise FoFError(-k, "fof_phase_times")
    return {names[i].decode(): (ms[i], ln[i]) for i in range(min(k, m))}


def fof_reset_times(h) -> int:
    return _check(load().fof_reset_times(h), "fof_reset_times")


def fof_kernel_launches(h) -> int:
    return load().fof_kernel_launches(h)


def fof_destroy(h) -> None:
    if h:
        load().fof_destroy(h)


def fof_run_noalloc(box, l_x, n, pos, ids, sizes, catalogue, cat_capacity, min_size, stream=None,
                    allow_capacity=False):
    """Allocation-free single-box run (see include/fof.h).  Returns
    (code, n_groups, n_cat)."""
    ng = ctypes.c_int64(0)
    nk = ctypes.c_int64(0)
    code = load().fof_run_noalloc(box, l_x, n, _ptr(pos), _ptr(ids), _ptr(sizes), _ptr(catalogue),
                                  cat_capacity, min_size, ctypes.byref(ng), ctypes.byref(nk),
                                  _stream(stream))
    if code != FOF_OK and not (allow_capacity and code == FOF_ERR_CAPACITY):
        raise FoFError(code, "fof_run_noalloc")
    return code, ng.value, nk.value


def fof_merge_links(a, b, query, weight_ids=None, weights=None, want_weights=False):
    """Union-find over gathered links (int64 numpy arrays); returns the
    smallest id of each query's merged set (and the set weights)."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    q = np.ascontiguousarray(query, dtype=np.int64)
    wi = np.ascontiguousarray(weight_ids if weight_ids is not None else np.zeros(0), dtype=np.int64)
    wv = np.ascontiguousarray(weights if weights is not None else np.zeros(0), dtype=np.int64)
    assert a.shape == b.shape and wi.shape == wv.shape
    lab = np.empty(q.shape[0], dtype=np.int64)
    wout = np.empty(q.shape[0], dtype=np.int64) if want_weights else None
    _check(load().fof_merge_links(a.shape[0], _ptr(a), _ptr(b), wi.shape[0], _ptr(wi), _ptr(wv),
                                  q.shape[0], _ptr(q), _ptr(lab), _ptr(wout) if wout is not None else None),
           "fof_merge_links")
    return (lab, wout) if want_weights else lab


# ---------------------------------------------------------------------------
# convenience wrappers over device tensors
# ---------------------------------------------------------------------------

class FoF:
    """One periodic box.  run(pos) -> (ids, sizes, catalogue[k, 2], n_groups)."""

    def __init__(self, box: float, l_x: float, n: int, opt: fof_options | None = None,
                 workspace=None):
        self.box, self.l_x, self.n = float(box), float(l_x), int(n)
        ws_bytes = 0
        if workspace is not None:
            ws_bytes = workspace.numel() * workspace.element_size()
        self.h = fof_create_ex(self.box, self.l_x, self.n, opt, workspace, ws_bytes)
        self.nbox = 1

    def close(self):
        if self.h:
            fof_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, pos, min_size: int = 1, cat_capacity: int | None = None, stream=None):
        import torch
        assert pos.is_cuda and pos.dtype == torch.float32 and pos.is_contiguous()
        dev = pos.device
        n = self.n
        if cat_capacity is None:
            cat_capacity = n
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        sizes = torch.empty(n, dtype=torch.int32, device=dev)
        cat = torch.empty((max(cat_capacity, 1), 2), dtype=torch.int32, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        fof_link(self.h, pos, s)
        _, ng, nk = fof_groups(self.h, ids, sizes, cat, cat_capacity, min_size, 1, s)
        return ids, sizes, cat[: min(nk[0], cat_capacity)], ng[0]


class FoFBatch:
    """Independent boxes in one plan; inputs and outputs concatenated."""

    def __init__(self, boxes, lxs, ns, opt: fof_options | None = None, workspace=None):
        self.ns = [int(v) for v in ns]
        self.nbox = len(self.ns)
        ws_bytes = 0
        if workspace is not None:
            ws_bytes = workspace.numel() * workspace.element_size()
        self.h = fof_batch_create(list(map(float, boxes)), list(map(float, lxs)), self.ns, opt,
                                  workspace, ws_bytes)

    def close(self):
        if self.h:
            fof_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, pos_concat, min_size: int = 1, cat_capacity: int | None = None, stream=None):
        import torch
        dev = pos_concat.device
        total = sum(self.ns)
        if cat_capacity is None:
            cat_capacity = total
        ids = torch.empty(total, dtype=torch.int32, device=dev)
        sizes = torch.empty(total, dtype=torch.int32, device=dev)
        cat = torch.empty((max(cat_capacity, 1), 2), dtype=torch.int32, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        fof_link(self.h, pos_concat, s)
        _, ng, nk = fof_groups(self.h, ids, sizes, cat, cat_capacity, min_size, self.nbox, s)
        return ids, sizes, cat[: min(sum(nk), cat_capacity)], ng, nk
