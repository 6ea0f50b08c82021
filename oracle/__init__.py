"""Plain FP64 CPU oracle for the contact-detection + STIV path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  It shares no code with the CUDA path.  The arithmetic lives in
``stiv_oracle.c`` (compiled with -ffp-contract=off); this module only loads it
and marshals numpy arrays.

Paper sections followed (arXiv 1812.04719): SH surface and quadrature grid
(Sec. 3.1.1), upsampling and triangulation (Sec. 3.1.2, Fig. 3), swept boxes
and bbiCheck (Sec. 3.3.1, Alg. 1), contact time (Eq. 3.1 with d_m = 0),
contact volume and its gradient (Eq. 3.2, App. A), ContactVolume (Alg. 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stiv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lp = ctypes.POINTER(ctypes.c_int64)
            L.orc_gl_nodes.argtypes = [ctypes.c_int, dp, dp]
            L.orc_legendre_norm.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            L.orc_legendre_norm.restype = None
            L.orc_synth.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_synth.restype = None
            L.orc_synth_vesicle.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_synth_vesicle.restype = None
            L.orc_mesh_fidelity.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_mesh_fidelity.restype = ctypes.c_double
            L.orc_mesh_point.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_mesh_point.restype = None
            L.orc_synth_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_synth_adjoint.restype = None
            L.orc_triangles.argtypes = [ctypes.c_int, ip]
            L.orc_edges.argtypes = [ctypes.c_int, ip]
            L.orc_vesicle_box.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
            L.orc_vesicle_box.restype = None
            L.orc_candidate_pairs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, ip]
            L.orc_candidate_pairs.restype = ctypes.c_int64
            L.orc_ccd_primitive.argtypes = [ctypes.c_int, dp, dp, dp]
            L.orc_stiv_primitive.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
            L.orc_stiv_primitive_v.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, dp]
            L.orc_ccd_primitive_dm.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp]
            L.orc_poly_roots01.argtypes = [dp, ctypes.c_int, dp]
            L.orc_contacts.argtypes = [ctypes.c_int, ip, lp, dp, ctypes.c_int64, ip, dp,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int64, ip, ip, ip, ip, dp, dp, dp, dp, dp, ip, ip, lp]
            L.orc_contacts.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _d(a):
    return _p(a, ctypes.c_double)


def _i(a):
    return _p(a, ctypes.c_int32)


def _l(a):
    return _p(a, ctypes.c_int64)


def nverts(P: int) -> int:
    return 2 * P * (P + 1) + 2


def ntris(P: int) -> int:
    return 4 * P * P + 4 * P


def nedges(P: int) -> int:
    return 6 * P * P + 6 * P


def gl_nodes(nq: int):
    x = np.zeros(nq); w = np.zeros(nq)
    lib().orc_gl_nodes(nq, _d(x), _d(w))
    return x, w


def legendre_norm(nmax: int, x: float) -> np.ndarray:
    out = np.zeros((nmax + 1) * (nmax + 2) // 2)
    lib().orc_legendre_norm(nmax, float(x), _d(out))
    return out


def synth(p: int, P: int, coef: np.ndarray) -> np.ndarray:
    """One scalar field: coef[(p+1)^2] -> values at the n_v(P) mesh vertices."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    assert coef.shape == ((p + 1) ** 2,)
    out = np.zeros(nverts(P))
    lib().orc_synth(p, P, _d(coef), _d(out))
    return out


def mesh_fidelity(p: int, P: int, coef: np.ndarray, X: np.ndarray, factor: int = 4) -> float:
    """Sec. 3.1.2 / Fig. 6: max over the order-(factor P) grid of the distance
    between the order-P triangle mesh (read in parameter space) and the smooth
    order-p surface.  coef [3][(p+1)^2] and X [3][n_v(P)] of one time level."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    assert coef.shape == (3, (p + 1) ** 2) and X.shape == (3, nverts(P))
    return float(lib().orc_mesh_fidelity(p, P, factor, _d(coef), _d(X)))


def mesh_point(P: int, X: np.ndarray, theta: float, phi: float) -> np.ndarray:
    """The order-P triangle mesh X [3][n_v(P)] at parameter (theta, phi)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_mesh_point(P, _d(X), float(theta), float(phi), _d(out))
    return out


def synth_vesicle(p: int, P: int, coef: np.ndarray) -> np.ndarray:
    """coef[2][3][(p+1)^2] -> X[2][3][n_v(P)]."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    assert coef.shape == (2, 3, (p + 1) ** 2)
    X = np.zeros((2, 3, nverts(P)))
    lib().orc_synth_vesicle(p, P, _d(coef), _d(X))
    return X


def synth_adjoint(p: int, P: int, g: np.ndarray) -> np.ndarray:
    """S^T g for one scalar field: g[n_v(P)] -> gcoef[(p+1)^2]."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert g.shape == (nverts(P),)
    out = np.zeros((p + 1) ** 2)
    lib().orc_synth_adjoint(p, P, _d(g), _d(out))
    return out


def triangles(P: int) -> np.ndarray:
    t = np.zeros((ntris(P), 3), dtype=np.int32)
    lib().orc_triangles(P, _i(t))
    return t


def edges(P: int) -> np.ndarray:
    e = np.zeros((nedges(P), 2), dtype=np.int32)
    n = lib().orc_edges(P, _i(e))
    assert n == nedges(P)
    return e


def vesicle_box(X: np.ndarray, dm: float = 0.0) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    b = np.zeros(6)
    lib().orc_vesicle_box(X.shape[-1], _d(X), float(dm), _d(b))
    return b


def candidate_pairs(boxes: np.ndarray, L) -> np.ndarray:
    """All (i<j, shift) pairs whose boxes overlap: rows (i, j, sx, sy, sz)."""
    boxes = np.ascontiguousarray(boxes, dtype=np.float64)
    Lv = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)))
    n = boxes.shape[0]
    cnt = lib().orc_candidate_pairs(n, _d(boxes), _d(Lv), 0, _i(np.zeros(5, np.int32)))
    out = np.zeros((max(cnt, 1), 5), dtype=np.int32)
    lib().orc_candidate_pairs(n, _d(boxes), _d(Lv), cnt, _i(out))
    return out[:cnt]


def ccd_primitive(kind: str, X0: np.ndarray, X1: np.ndarray):
    """Single primitive pair.  kind 'vf' (points xp, x0, x1, x2) or 'ee'
    (p0, p1, q0, q1).  Returns (status, tau, w1, w2); status 1 = contact,
    2 = degenerate, 0 = none."""
    X0 = np.ascontiguousarray(X0, dtype=np.float64).reshape(4, 3)
    X1 = np.ascontiguousarray(X1, dtype=np.float64).reshape(4, 3)
    out = np.zeros(3)
    st = lib().orc_ccd_primitive(0 if kind == "vf" else 1, _d(X0), _d(X1), _d(out))
    return st, out[0], out[1], out[2]


def stiv_primitive(kind: str, X0, X1, eps_dt: float):
    """V_k and dV_k/dX1 [4][3] of one primitive pair (0 if no contact)."""
    X0 = np.ascontiguousarray(X0, dtype=np.float64).reshape(4, 3)
    X1 = np.ascontiguousarray(X1, dtype=np.float64).reshape(4, 3)
    out = np.zeros(13)
    st = lib().orc_stiv_primitive(0 if kind == "vf" else 1, _d(X0), _d(X1), float(eps_dt), _d(out))
    return st, out[0], out[1:].reshape(4, 3)


class Contacts(dict):
    """Contact list of a scene: numpy arrays keyed by name."""


def contacts(P_ves, X_list_or_flat, pairs, L, eps_dt: float, prune: bool = True,
             include_ee: bool = True, grad: bool = True, nthreads: int = 0, voff=None,
             velocity: str = "relative", grad_wrt: str = "X1", d_m: float = 0.0):
    """Alg. 2 checkContact over candidate vesicle pairs.

    P_ves: grid order per vesicle.  X: either a list of [2][3][n_v] arrays or
    a flat float64 array with offsets ``voff``.  pairs: rows (i, j, sx, sy, sz).
    Returns a dict: pair, type, a, b, tau, w[.,2], V (per contact), V_pair (per
    pair row), grad [.,4,3], gves/gvid [.,4], counts (contacts, prim pairs
    tested, degenerate, floating-point operations of the contact tests).
    velocity "absolute" takes U_k as the contact point's own velocity (the
    literal reading); grad_wrt "X0" differentiates with respect to X0; d_m > 0
    uses the degree-six test of Eq. 3.1 (contact within d_m) and widens the
    second vesicle's primitive boxes by d_m."""
    assert velocity in ("relative", "absolute") and grad_wrt in ("X1", "X0")
    P_ves = np.ascontiguousarray(P_ves, dtype=np.int32)
    if voff is None:
        sizes = [6 * nverts(int(P)) for P in P_ves]
        voff = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        flat = np.concatenate([np.ascontiguousarray(x, dtype=np.float64).ravel() for x in X_list_or_flat])
    else:
        voff = np.ascontiguousarray(voff, dtype=np.int64)
        flat = np.ascontiguousarray(X_list_or_flat, dtype=np.float64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 5)
    Lv = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)))
    npairs = pairs.shape[0]
    counts = np.zeros(4, dtype=np.int64)
    V_pair = np.zeros(max(npairs, 1))
    L_ = lib()
    args_head = (len(P_ves), _i(P_ves), _l(voff), _d(flat), npairs, _i(pairs if npairs else np.zeros((1, 5), np.int32)),
                 _d(Lv), int(prune), int(include_ee), float(d_m), float(eps_dt), int(velocity == "absolute"),
                 int(grad_wrt == "X0"), int(nthreads))

    def run(cap):
        c = max(cap, 1)
        o = dict(pair=np.zeros(c, np.int32), type=np.zeros(c, np.int32), a=np.zeros(c, np.int32),
                 b=np.zeros(c, np.int32), tau=np.zeros(c), w=np.zeros((c, 2)), V=np.zeros(c),
                 grad=np.zeros((c, 4, 3)) if grad else None, gves=np.zeros((c, 4), np.int32),
                 gvid=np.zeros((c, 4), np.int32))
        n = L_.orc_contacts(*args_head, cap, _i(o["pair"]), _i(o["type"]), _i(o["a"]), _i(o["b"]),
                            _d(o["tau"]), _d(o["w"]), _d(o["V"]), _d(V_pair),
                            _d(o["grad"]) if grad else None, _i(o["gves"]), _i(o["gvid"]), _l(counts))
        return n, o

    n, o = run(4096)
    if n > 4096:
        n, o = run(n)
    out = Contacts({k: (v[:n] if v is not None else None) for k, v in o.items()})
    out["V_pair"] = V_pair[:npairs].copy()
    out["counts"] = counts.copy()
    return out


def stiv_primitive_variant(kind: str, X0, X1, eps_dt: float, velocity: str = "relative", grad_wrt: str = "X1",
                           d_m: float = 0.0):
    """stiv_primitive with the literal velocity reading, the gradient with
    respect to X0 and/or d_m > 0 (the degree-six contact time)."""
    X0 = np.ascontiguousarray(X0, dtype=np.float64).reshape(4, 3)
    X1 = np.ascontiguousarray(X1, dtype=np.float64).reshape(4, 3)
    out = np.zeros(13)
    st = lib().orc_stiv_primitive_v(0 if kind == "vf" else 1, _d(X0), _d(X1), float(eps_dt), float(d_m),
                                    int(velocity == "absolute"), int(grad_wrt == "X0"), _d(out))
    return st, out[0], out[1:].reshape(4, 3)


def ccd_primitive_dm(kind: str, X0, X1, d_m: float):
    """Single primitive pair with minimum separation d_m (Eq. 3.1, degree six
    for d_m > 0).  Returns (status, tau, w1, w2)."""
    X0 = np.ascontiguousarray(X0, dtype=np.float64).reshape(4, 3)
    X1 = np.ascontiguousarray(X1, dtype=np.float64).reshape(4, 3)
    out = np.zeros(3)
    st = lib().orc_ccd_primitive_dm(0 if kind == "vf" else 1, _d(X0), _d(X1), float(d_m), _d(out))
    return st, out[0], out[1], out[2]


def poly_roots01(c) -> np.ndarray:
    """Roots in (0, 1) of the polynomial c[0] + c[1] t + ... (degree <= 6),
    ascending, by the derivative-chain isolation of the d_m > 0 test."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.zeros(6)
    n = lib().orc_poly_roots01(_d(c), len(c) - 1, _d(out))
    return out[:n].copy()
