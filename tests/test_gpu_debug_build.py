"""The bounds-checked build (libfof_gb300_debug.so, FOF_DEBUG_CHECKS) gives
the oracle's answer and reports no bad slot on inputs that reach every link
kernel: clustered boxes with team, dense and big cells, and a batch.

Runs in a child process, because the library is chosen when the binding
loads it (FOF_LIBRARY=debug)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import oracle
from paper_2003_11468_gb300 import fof, synth
assert fof.LIB_PATH.endswith("libfof_gb300_debug.so"), fof.LIB_PATH
cases = []
n, box = 300000, 30.0
cases.append((synth.clustered_box(n, box, 120, seed=123), box, synth.linking_length(n, box, 0.25), None))
import test_gpu_parity as t
pos, bx, lx, nc = t._big_cell_box(7)
opt = fof.fof_options(); opt.cells_per_axis = nc; opt.brick_cells = 2
cases.append((pos, bx, lx, opt))
for pos, bx, lx, opt in cases:
    with fof.FoF(bx, lx, pos.shape[0], opt) as f:       # raises on FOF_ERR_INTERNAL
        ids, sizes, _, _ = f.run(torch.from_numpy(pos).cuda())
    wid, wsz = oracle.groups(pos, bx, lx)
    assert np.array_equal(ids.cpu().numpy(), wid)
    assert np.array_equal(sizes.cpu().numpy(), wsz)
print("debug build ok")
'''


def test_debug_build_parity():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_11468_gb300 import build
    if not os.path.exists(build.DEBUG_LIB):
        build.build(debug=True)
    env = dict(os.environ, FOF_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "debug build ok" in r.stdout
