"""Oracle synthesis of a scene's vertices for the parity tests, spread over
host threads (the oracle's C routines run without the interpreter lock; no
process is forked).  Test infrastructure only: the vertices the CUDA path is
checked on come from the oracle, never from the CUDA path's own upsampling."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle

_cache = {}


def _synth(args):
    p, P, coef = args
    return oracle.synth_vesicle(p, P, coef).ravel()


def oracle_vertices(sc, workers=None) -> np.ndarray:
    """Flat FP64 vertices of every vesicle in the library's vertex layout
    (per vesicle [2][3][n_v], at sc.vert_off()), synthesised by the oracle
    (Sec. 2, the SH expansion evaluated on the upsampled grid and poles)."""
    key = (sc.name, sc.n, float(np.asarray(sc.coef).sum()))
    if key in _cache:
        return _cache[key]
    oracle.build()
    args = [(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    if sc.n <= 32:
        parts = [_synth(a) for a in args]
    else:
        nw = workers or max(1, min(os.cpu_count() or 1, 32))
        with ThreadPoolExecutor(nw) as ex:
            parts = list(ex.map(_synth, args))
    flat = np.concatenate(parts)
    assert flat.size == sc.n_vert_values()
    _cache[key] = flat
    return flat
