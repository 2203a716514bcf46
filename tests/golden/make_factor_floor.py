"""Writes tests/golden/factor_floor.json: sum_i nnz(L_i) of the local Cholesky factors
of Algorithm 1 under a fill-reducing order, for the benchmark workloads.

    python tests/golden/make_factor_floor.py [c1 c2 c3 c4]

Every number comes from the oracle alone (oracle.partition, oracle.algmortar's local
matrices A_i of Eq. (A_i), oracle.symbolic's count) on the seeded inputs of synth.py.
The count is the byte floor of the per-iteration local solves: each of the two
triangular sweeps reads every entry of every L_i once.
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import algmortar as oa  # noqa: E402
from oracle import partition as op  # noqa: E402
from oracle import symbolic as osym  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "factor_floor.json")
CONFIGS = {"c1": synth.config1, "c2": synth.config2, "c3": synth.config3, "c4": synth.config4}


def _count(Ai):
    return osym.factor_nnz(Ai, osym.fill_reducing_order(Ai))


def partition_sha1(part):
    return hashlib.sha1(np.ascontiguousarray(part, dtype=np.int32).tobytes()).hexdigest()


def floor_of(name, pool):
    P = CONFIGS[name]()
    t = time.time()
    part = op.partition(P.A, P.part_sizes)
    sk = oa.skeleton(P.A, part)
    A_loc = oa.local_matrices(sk)
    counts = pool.map(_count, A_loc, chunksize=8)
    return {
        "workload": P.name,
        "n": int(P.n),
        "n_parts": int(P.n_parts),
        "partition_sha1": partition_sha1(part),
        "sum_nnz_L": int(sum(counts)),
        "max_nnz_L": int(max(counts)),
        "order": "multiple minimum degree on A_i + A_i^T (SuperLU), symbolic elimination",
        "seconds": round(time.time() - t, 1),
    }


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        for name in names:
            data[name] = floor_of(name, pool)
            print(name, data[name], flush=True)
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c2", "c3", "c4"])
