"""Writes narrow_ops_per_pair.json: the algorithmic work of the narrow phase
per unit, i.e. the floating-point operations of the Eq. 3.1 contact test
(d_m = 0: cubic, root isolation, inside test) per primitive pair whose exact
swept boxes overlap, counted by the oracle on the 144-vesicle piece of the
58% lattice workload (p = 16 -> 32, periodic box).

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


def main():
    oracle.build()
    sc = G.scene_lattice58((6, 6, 2))
    Xs = [oracle.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    boxes = np.stack([oracle.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = oracle.candidate_pairs(boxes, sc.L)
    t0 = time.time()
    c = oracle.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=False)
    n_contacts, n_prim, n_degen, n_ops = (int(x) for x in c["counts"])
    out = {
        "scene": sc.name,
        "candidate_pairs": int(len(pairs)),
        "prim_pairs": n_prim,
        "contacts": n_contacts,
        "degenerate": n_degen,
        "ops": n_ops,
        "ops_per_prim_pair": n_ops / n_prim,
        "counting": "+ - * / sqrt = 1, fma = 2, negation and comparison 0",
    }
    with open(os.path.join(HERE, "narrow_ops_per_pair.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out), f"{time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
