#!/usr/bin/env python3
"""Write the golden topology records of the benchmarked graphs.

Calls only the CPU oracle (``oracle.Graph``: Eq. 4 mipmap, Sec. 3.2-3.3
factorisation with the balanced positional pairing, Sec. 3.4 levels and the
canonical numbering) on the volumes of the seeded host generators.  Nothing
here runs on or reads from the GPU path.  For each configuration the record
holds the sizes (N, S, D, L, per-level dims), the depth bucket offsets, the
longest mixture and the pair count, and sha256 digests of the node table
(p, q uint32; a, b uint64, canonical order) and of the node ID of every voxel
of every mip level (uint32, x fastest), all little-endian, and the size and
sha256 of the graph's bitstream (Table 1, oracle.Graph.bitstream).

    python tests/golden/make_graph_goldens.py 2 4 [3]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_02702_gb300 import synth  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def record(cfg_index: int) -> dict:
    cfg = synth.CONFIGS[cfg_index]
    t0 = time.perf_counter()
    vol = synth.make_volume(cfg_index)
    t1 = time.perf_counter()
    g = oracle.Graph(vol, cfg["S"])
    t2 = time.perf_counter()
    N = g.N
    rec = {
        "config": cfg_index, "workload": cfg["name"], "dims": list(cfg["dims"]), "S": cfg["S"],
        "N": N, "D": g.D, "L": g.L, "level_dims": g.dims.tolist(), "bucket": g.bucket.tolist(),
        "max_list": g.max_nnz, "pairs": g.pairs,
        "sha256": {"p": digest(g.p[:N]), "q": digest(g.q[:N]), "a": digest(g.a[:N]), "b": digest(g.b[:N]),
                   "mip": [digest(g.mip(l)) for l in range(g.L)]},
        "bitstream": {},
        "source": "oracle.Graph on synth.make_volume(%d) (host generator)" % cfg_index,
    }
    stream = g.bitstream()
    rec["bitstream"] = {"bytes": len(stream), "sha256": hashlib.sha256(stream).hexdigest()}
    g.close()
    print("cfg %d: volume %.1f s, oracle build %.1f s, N=%d D=%d" % (cfg_index, t1 - t0, t2 - t1, N, rec["D"]),
          flush=True)
    return rec


def main(argv):
    cfgs = [int(a) for a in argv] or [2, 4]
    for c in cfgs:
        rec = record(c)
        with open(os.path.join(HERE, "graph_cfg%d.json" % c), "w") as f:
            json.dump(rec, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
