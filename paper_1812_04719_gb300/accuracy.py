"""The precision (MIXED) form's stated accuracy against the FP64 form.

The MIXED form synthesises the vertices with split (3xTF32) products on the
tensor cores and stores them as FP32; the broad phase, the contact test
(Eq. 3.1), V (Eq. 3.2) and dV/dX1 then run in FP64 on those vertices.  Its
error against the FP64 form therefore comes from the vertex error alone,
which is bounded per coordinate of field (vesicle, time, coordinate), with SH
coefficients a_q of order p, by

    delta = 2^-23 |X| + 2^-19 sum_{q>0} |a_q| sqrt((2p + 1) / (2 pi))

(each split product keeps a relative error near 2^-22; FP32 accumulation and
the final rounding to FP32 add the rest).  delta_k below is the largest delta
over the four points of contact k, both time levels and all coordinates.

Propagated to the outputs (first order in delta; the GPU tests assert each
on the 1440-vesicle workload):

1. A contact present in both forms has
       |V_mixed - V_fp64| <= S_k delta_k,
   S_k = ||dV_k/dX1||_1 + ||dV_k/dX0||_1 (all 24 coordinates of its points):
   the first-order change of V_k under coordinate errors of at most delta_k.
2. A contact whose decision margins exceed MARGIN_FACTOR delta_k is present
   in both forms.  The margins, in length units, at the contact time:
     - inside test: the distance of the contact point from the nearest edge
       line of the triangle (VF), or of the closest points from the nearer
       end of their edge times the sine of the edges' angle (EE), divided by
       1 + v_t / v_n;
     - contact time: min(tau, 1 - tau) v_n;
   v_n and v_t are the normal and tangential parts of the relative
   displacement of the two contact points over the step.  Moving every point
   by at most delta per coordinate (sqrt(3) delta in length) moves a contact
   point relative to an edge line, or to the other primitive's plane, by at
   most 2 sqrt(3) delta, and shifts the contact time by that over v_n, which
   slides the contact point by that times v_t / v_n; 2 sqrt(3) < 4 =
   MARGIN_FACTOR.  Every contact in only one form's list is therefore a
   marginal one.
3. The gradient row of a contact present in both forms has
       ||g_mixed - g_fp64||_inf <= GRAD_FACTOR kappa_k ||g_fp64||_inf,
   kappa_k = S_k delta_k / V_k (the first-order relative change of V_k).
   The second derivatives of V_k scale like its first derivatives over the
   same length scales, so the relative change of the row follows kappa_k;
   the constant is not derived: GRAD_FACTOR = 4 is four times the largest
   ratio measured on the 1440-vesicle workload (0.91).
4. Per vesicle pair, by the triangle inequality and (1):
       |V_pair,mixed - V_pair,fp64| <= sum_{k in both} S_k delta_k
                                       + sum_{k in one list only} V_k.

This module evaluates these quantities on host arrays (numpy); it is a
diagnostic of the library's results, not a step of the path.
"""
from __future__ import annotations

import math

import numpy as np

MARGIN_FACTOR = 4.0
GRAD_FACTOR = 4.0


def vertex_delta(p: int, coef: np.ndarray, X: np.ndarray) -> np.ndarray:
    """delta per coordinate of one vesicle: coef [2][3][(p+1)^2], X [2][3][n_v]
    (the FP64 vertices) -> [2][3][n_v]."""
    a1 = np.abs(np.asarray(coef)[:, :, 1:]).sum(axis=-1)[:, :, None]
    return 2.0 ** -23 * np.abs(X) + 2.0 ** -19 * a1 * math.sqrt((2 * p + 1) / (2 * math.pi))


def point_delta(p, coef_of, vert_off, X_flat) -> np.ndarray:
    """Per vertex of the scene (index vert_off[v] // 6 + vertex id), the largest
    delta over both time levels and the three coordinates.  p: orders per
    vesicle; coef_of(v): its coefficients [2][3][(p+1)^2]; X_flat: the FP64
    vertices in the library's layout."""
    out = np.zeros(len(X_flat) // 6)
    for v in range(len(p)):
        o = int(vert_off[v])
        nv = (2 * int(p[v])) * (2 * int(p[v]) + 1) * 2 + 2
        X = np.asarray(X_flat[o:o + 6 * nv], dtype=np.float64).reshape(2, 3, nv)
        out[o // 6:o // 6 + nv] = vertex_delta(int(p[v]), coef_of(v), X).max(axis=(0, 1))
    return out


def shift_vec(code):
    code = np.asarray(code)
    return np.stack([code // 9 - 1, (code // 3) % 3 - 1, code % 3 - 1], axis=-1)


def contact_points(r: dict, X_flat, vert_off, L):
    """Positions [n][4][3] at t_n and t_{n+1} of each contact's four points
    (in the order of the contact test: VF vertex then triangle, EE p0 p1 q0
    q1), the second vesicle's points at the pair's periodic image.  r: one
    step's results as numpy arrays (i, j, shift, pair, gves, gvid)."""
    gves, gvid = np.asarray(r["gves"], np.int64), np.asarray(r["gvid"], np.int64)
    pair = np.asarray(r["pair"], np.int64)
    j = np.asarray(r["j"], np.int64)[pair]
    sh = shift_vec(np.asarray(r["shift"])[pair]) * np.asarray(L, dtype=np.float64)
    vo = np.asarray(vert_off, np.int64)[gves]
    nv = (np.diff(np.append(np.asarray(vert_off, np.int64), len(X_flat))) // 6)[gves]
    X = np.asarray(X_flat, dtype=np.float64)
    X0 = np.stack([X[vo + c * nv + gvid] for c in range(3)], axis=-1)
    X1 = np.stack([X[vo + (3 + c) * nv + gvid] for c in range(3)], axis=-1)
    onj = (gves == j[:, None])[:, :, None]
    return X0 + onj * sh[:, None, :], X1 + onj * sh[:, None, :]


def margins(typ, X0, X1, tau, w):
    """Decision margins (length units) of contacts: (inside margin, time
    margin, v_n, v_t), see the module docstring.  typ: 0/1 VF, 2 EE; X0, X1
    [n][4][3]; tau [n]; w [n][2] (barycentric weights b1, b2 or s, u)."""
    typ = np.asarray(typ)
    tau = np.asarray(tau, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    D = X1 - X0
    Y = X0 + tau[:, None, None] * D
    vf = (typ < 2)[:, None]
    a = np.where(vf, Y[:, 2] - Y[:, 1], Y[:, 1] - Y[:, 0])
    b = np.where(vf, Y[:, 3] - Y[:, 1], Y[:, 3] - Y[:, 2])
    m = np.cross(a, b)
    mn = np.maximum(np.linalg.norm(m, axis=1), 1e-300)
    w1, w2 = w[:, 0], w[:, 1]
    w0 = 1.0 - w1 - w2
    d_vf = D[:, 0] - (w0[:, None] * D[:, 1] + w1[:, None] * D[:, 2] + w2[:, None] * D[:, 3])
    d_ee = (D[:, 2] + w2[:, None] * (D[:, 3] - D[:, 2])) - (D[:, 0] + w1[:, None] * (D[:, 1] - D[:, 0]))
    rel = np.where(vf, d_vf, d_ee)
    nh = m / mn[:, None]
    rn = (rel * nh).sum(axis=1)
    vn = np.abs(rn)
    vt = np.linalg.norm(rel - rn[:, None] * nh, axis=1)
    # VF: weight times the altitude over the edge opposite each vertex
    e0 = np.linalg.norm(Y[:, 3] - Y[:, 2], axis=1)
    e1 = np.linalg.norm(Y[:, 3] - Y[:, 1], axis=1)
    e2 = np.linalg.norm(Y[:, 2] - Y[:, 1], axis=1)
    m_vf = np.minimum(np.minimum(w0 * mn / e0, w1 * mn / e1), w2 * mn / e2)
    la, lb = np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1)
    sin = mn / np.maximum(la * lb, 1e-300)
    m_ee = np.minimum(np.minimum(w1, 1.0 - w1) * la, np.minimum(w2, 1.0 - w2) * lb) * sin
    inside = np.where(typ < 2, m_vf, m_ee)
    tmarg = np.minimum(tau, 1.0 - tau) * vn
    return inside, tmarg, vn, vt


def scaled_margin(inside, tmarg, vn, vt, delta):
    """min(inside / (delta (1 + v_t / v_n)), time margin / delta): the
    contact's margin in units of its vertex bound."""
    amp = 1.0 + vt / np.maximum(vn, 1e-300)
    return np.minimum(inside / (delta * amp), tmarg / delta)


def contact_keys(r: dict) -> np.ndarray:
    """One int64 key per contact: (i, j, shift, type, a, b)."""
    pair = np.asarray(r["pair"], np.int64)
    i = np.asarray(r["i"], np.int64)[pair]
    j = np.asarray(r["j"], np.int64)[pair]
    s = np.asarray(r["shift"], np.int64)[pair]
    return ((((i << 13) | j) << 5 | s) << 32) | (np.asarray(r["type"], np.int64) << 30) | \
        (np.asarray(r["a"], np.int64) << 15) | np.asarray(r["b"], np.int64)


def compare(ra: dict, Xa, rb: dict, Xb, grad_x0_b, pdelta, vert_off, L) -> dict:
    """The MIXED results ra (on its vertices Xa) against the FP64 results rb
    (on Xb, with dV/dX0 rows grad_x0_b), both numpy dicts of one step
    (i, j, shift, pair, type, a, b, tau, w, V, V_pair, grad, gves, gvid);
    pdelta: point_delta of the scene.  Returns the figures of bounds 1-4 and
    whether each holds."""
    ka, kb = contact_keys(ra), contact_keys(rb)
    _, ia, ib = np.intersect1d(ka, kb, assume_unique=True, return_indices=True)
    only_a = np.setdiff1d(np.arange(len(ka)), ia)
    only_b = np.setdiff1d(np.arange(len(kb)), ib)
    nb = len(kb)
    g1 = np.asarray(rb["grad"]).reshape(nb, -1)
    g0 = np.asarray(grad_x0_b).reshape(nb, -1)
    vo6 = np.asarray(vert_off, np.int64) // 6
    dk_b = pdelta[vo6[np.asarray(rb["gves"], np.int64)] + np.asarray(rb["gvid"], np.int64)].max(axis=1)
    dk_a = pdelta[vo6[np.asarray(ra["gves"], np.int64)] + np.asarray(ra["gvid"], np.int64)].max(axis=1)
    S = np.abs(g1).sum(axis=1) + np.abs(g0).sum(axis=1)
    Va, Vb = np.asarray(ra["V"])[ia], np.asarray(rb["V"])[ib]
    bnd = S[ib] * dk_b[ib]
    v_ratio = np.abs(Va - Vb) / np.maximum(bnd, 1e-300)
    kappa = bnd / np.maximum(Vb, 1e-300)
    ga = np.asarray(ra["grad"]).reshape(len(ka), -1)[ia]
    gb = g1[ib]
    g_rel = np.abs(ga - gb).max(axis=1) / np.maximum(np.abs(gb).max(axis=1), 1e-300)
    g_ratio = g_rel / np.maximum(kappa, 1e-300)

    def scaled(r, X, idx, dk):
        if len(idx) == 0:
            return np.zeros(0)
        sub = {k: (np.asarray(v)[idx] if k in ("pair", "gves", "gvid") else v) for k, v in r.items()}
        X0, X1 = contact_points(sub, X, vert_off, L)
        ins, tm, vn, vt = margins(np.asarray(r["type"])[idx], X0, X1, np.asarray(r["tau"])[idx],
                                  np.asarray(r["w"])[idx])
        return scaled_margin(ins, tm, vn, vt, dk[idx])

    mu_a, mu_b = scaled(ra, Xa, only_a, dk_a), scaled(rb, Xb, only_b, dk_b)
    mu_sym = np.concatenate([mu_a, mu_b])
    # bound 4 per vesicle pair (pairs keyed by (i, j, shift))
    def pkeys(r):
        return (((np.asarray(r["i"], np.int64) << 13) | np.asarray(r["j"], np.int64)) << 5) | \
            np.asarray(r["shift"], np.int64)
    pa, pb = pkeys(ra), pkeys(rb)
    Vpa, Vpb = np.asarray(ra["V_pair"]), np.asarray(rb["V_pair"])
    allp = np.union1d(pa, pb)
    ea = np.zeros(len(allp)); eb = np.zeros(len(allp))
    ea[np.searchsorted(allp, pa)] = Vpa
    eb[np.searchsorted(allp, pb)] = Vpb
    pidx_b = np.searchsorted(allp, pb)[np.asarray(rb["pair"], np.int64)]
    pidx_a = np.searchsorted(allp, pa)[np.asarray(ra["pair"], np.int64)]
    pbound = np.zeros(len(allp))
    np.add.at(pbound, pidx_b[ib], bnd)
    np.add.at(pbound, pidx_b[only_b], np.asarray(rb["V"])[only_b])
    np.add.at(pbound, pidx_a[only_a], np.asarray(ra["V"])[only_a])
    dvp = np.abs(ea - eb)
    out = {
        "contacts_fp64": int(nb), "contacts_mixed": int(len(ka)), "contacts_both": int(len(ia)),
        "only_mixed": int(len(only_a)), "only_fp64": int(len(only_b)),
        "V_ratio_max": float(v_ratio.max()) if len(ia) else 0.0,
        "grad_rel_max": float(g_rel.max()) if len(ia) else 0.0,
        "grad_ratio_max": float(g_ratio.max()) if len(ia) else 0.0,
        "symdiff_margin_max": float(mu_sym.max()) if len(mu_sym) else 0.0,
        "symdiff_volume": float(np.asarray(ra["V"])[only_a].sum() + np.asarray(rb["V"])[only_b].sum()),
        "pair_ratio_max": float((dvp / np.maximum(pbound, 1e-300))[pbound > 0].max()) if (pbound > 0).any() else 0.0,
        "pairs_exceeding_bound": int((dvp > pbound * (1 + 1e-12) + 1e-300).sum()),
        "V_pair_abs_err_sum_over_V_sum": float(dvp.sum() / max(eb.sum(), 1e-300)),
        "V_pair_rel_err_max": float((dvp / np.maximum(eb, 1e-300))[eb > 0].max()) if (eb > 0).any() else 0.0,
        "delta_max": float(pdelta.max()),
    }
    out["bound1_V_holds"] = out["V_ratio_max"] <= 1.0
    out["bound2_lists_hold"] = out["symdiff_margin_max"] <= MARGIN_FACTOR
    out["bound3_grad_holds"] = out["grad_ratio_max"] <= GRAD_FACTOR
    out["bound4_pairs_hold"] = out["pairs_exceeding_bound"] == 0
    return out
