"""Write the full-size parity goldens: SHA-256 of the oracle's outputs.

Calls only the seeded generators (paper_2003_11468_gb300.synth, which holds
no group-finder arithmetic) and the CPU oracle (oracle/), never the CUDA
library.  For every workload it stores the SHA-256 of the float32 input (so
a test can tell a generator difference from a group-finder difference), of
the int32 ids and sizes arrays, of the int32 catalogue rows (label, size),
and the group and catalogue counts.  The GPU tests recompute the same
hashes from the library's outputs, which compares every element bit for bit.

  python tests/golden/make_fullsize_goldens.py small     # 32^3 uniform, 256^3 clustered
  python tests/golden/make_fullsize_goldens.py batch     # the 512 boxes of the batched form
  python tests/golden/make_fullsize_goldens.py served    # the served workload's input pool
  python tests/golden/make_fullsize_goldens.py 1024      # the 1024^3 box (about 52 GB of RAM)

Records go to tests/golden/fullsize/<set>.json.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "fullsize")


def sha(a) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def record(name, pos, box, l_x, min_size, extra=None):
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    ids, sizes = oracle.groups(pos, box, l_x)
    cat = oracle.catalogue(sizes, min_size)
    dt = time.perf_counter() - t0
    rec = {"name": name, "n": int(pos.shape[0]), "box": box, "l_x": l_x, "min_size": min_size,
           "input_sha256": sha(pos), "ids_sha256": sha(ids.astype("<i4")),
           "sizes_sha256": sha(sizes.astype("<i4")), "catalogue_sha256": sha(cat.astype("<i4")),
           "n_groups": int(np.count_nonzero(sizes)), "n_catalogue": int(cat.shape[0]),
           "largest_group": int(sizes.max()) if sizes.size else 0, "oracle_s": round(dt, 2)}
    if extra:
        rec.update(extra)
    return rec


def _batch_one(b):
    from paper_2003_11468_gb300 import synth
    sp = synth.batch_512()[b]
    pos = synth.make_batch_box(sp)
    return record(f"batch-512/box-{b}", pos, sp["box"], sp["l_x"], sp["min_size"],
                  {"box_index": b, "seed": sp["seed"]})


def _served_one(k):
    from paper_2003_11468_gb300 import synth
    sp = synth.served_pool()[k]
    pos = synth.make_served(sp)
    return record(f"served-pool/{k}", pos, sp["box"], sp["l_x"], sp["min_size"],
                  {"pool_index": k, "seed": sp["seed"]})


def _named(which):
    from paper_2003_11468_gb300 import synth
    c = {"32k": synth.uniform_32k, "256": synth.clustered_256, "1024": synth.clustered_1024}[which]()
    pos = c["make"]()
    return record(c["name"], pos, c["box"], c["l_x"], c["min_size"], {"seed": c["seed"]})


def write(set_name, recs, arg):
    os.makedirs(OUT, exist_ok=True)
    doc = {"generated_by": "tests/golden/make_fullsize_goldens.py " + arg,
           "machine": platform.machine(), "records": recs}
    path = os.path.join(OUT, f"{set_name}.json")
    with open(path + ".tmp", "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    os.replace(path + ".tmp", path)
    print(f"wrote {path}: {len(recs)} records", flush=True)


def main(argv):
    which = argv[1] if len(argv) > 1 else "small"
    import oracle
    oracle.build()
    procs = int(os.environ.get("GOLDEN_PROCS", str(os.cpu_count() or 1)))
    if which == "small":
        write("small", [_named("32k"), _named("256")], which)
    elif which == "1024":
        write("clustered_1024", [_named("1024")], which)
    elif which in ("batch", "served"):
        from paper_2003_11468_gb300 import synth
        count = len(synth.batch_512()) if which == "batch" else len(synth.served_pool())
        fn = _batch_one if which == "batch" else _served_one
        # largest first, so the long ones do not end up last on one worker
        if which == "batch":
            order = sorted(range(count), key=lambda b: -synth.batch_512()[b]["n"])
        else:
            order = list(range(count - 1, -1, -1))
        with mp.get_context("spawn").Pool(procs) as pool:
            recs = pool.map(fn, order, chunksize=1)
        recs.sort(key=lambda r: r.get("box_index", r.get("pool_index")))
        write("batch_512" if which == "batch" else "served_pool", recs, which)
    else:
        raise SystemExit(f"unknown set {which!r}")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
