"""Test helper: run the oracle over a whole Scene (Alg. 2 with all-pairs box
tests), returning numpy arrays.  Test infrastructure only."""
import numpy as np

import oracle as O


def synth_scene(sc):
    return [O.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]


def flat_verts(sc, Xs):
    return np.concatenate([X.ravel() for X in Xs])


def run_scene(sc, Xs=None, prune=True, include_ee=True, grad=True, nthreads=0, pairs=None):
    if Xs is None:
        Xs = synth_scene(sc)
    boxes = np.stack([O.vesicle_box(X, sc.d_m) for X in Xs])
    if pairs is None:
        pairs = O.candidate_pairs(boxes, sc.L)
    c = O.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, prune=prune, include_ee=include_ee,
                   grad=grad, nthreads=nthreads)
    c["pairs"] = pairs
    c["boxes"] = boxes
    return Xs, c


def contact_keys(c, pairs=None):
    """Set of (i, j, sx, sy, sz, type, a, b) tuples."""
    pr = c["pairs"] if pairs is None else pairs
    return {tuple(int(x) for x in pr[c["pair"][k]]) + (int(c["type"][k]), int(c["a"][k]), int(c["b"][k]))
            for k in range(len(c["pair"]))}
