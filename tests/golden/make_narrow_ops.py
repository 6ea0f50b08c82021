"""Writes narrow_ops_per_pair.json: the algorithmic work of the narrow phase
per unit, i.e. the floating-point operations of the Eq. 3.1 contact test
(d_m = 0: cubic, root isolation, inside test) per primitive pair whose exact
swept boxes overlap, counted by the oracle, for each benchmark workload:

  1440  the 144-vesicle piece of the 58% lattice (same cells, density, step
        and order), every candidate pair;
  4096  a seeded random sample of 200 candidate pairs of the 4096-vesicle
        40% workload (orders 8, 12, 16);
  256   every candidate pair of the 256-vesicle 50% workload;
  64    every candidate pair of the 64-vesicle 30% workload.

Calls only the oracle (and the seeded scene generator for its inputs):
    python tests/golden/make_narrow_ops.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1812_04719_gb300 import scenegen as G  # noqa: E402


def count(sc, sample=None, seed=0):
    Xs = [oracle.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    boxes = np.stack([oracle.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = oracle.candidate_pairs(boxes, sc.L)
    rows = pairs
    if sample is not None and len(pairs) > sample:
        rng = np.random.default_rng(seed)
        rows = pairs[np.sort(rng.choice(len(pairs), sample, replace=False))]
    t0 = time.time()
    c = oracle.contacts(sc.P, Xs, rows, sc.L, sc.eps * sc.dt, grad=False)
    n_contacts, n_prim, n_degen, n_ops = (int(x) for x in c["counts"])
    return {
        "scene": sc.name,
        "candidate_pairs": int(len(pairs)),
        "pairs_counted": int(len(rows)),
        "prim_pairs": n_prim,
        "contacts": n_contacts,
        "degenerate": n_degen,
        "ops": n_ops,
        "ops_per_prim_pair": n_ops / n_prim,
        "oracle_seconds": round(time.time() - t0, 1),
    }


def main():
    oracle.build()
    out = {
        "counting": "+ - * / sqrt = 1, fma = 2, negation and comparison 0",
        "workloads": {
            "1440": count(G.scene_lattice58((6, 6, 2))),
            "4096": count(G.scene_4096(), sample=200, seed=4096),
            "256": count(G.scene_256()),
            "64": count(G.scene_64()),
        },
    }
    with open(os.path.join(HERE, "narrow_ops_per_pair.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
