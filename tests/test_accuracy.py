"""Host-side checks of the MIXED form's accuracy evaluation
(paper_1812_04719_gb300/accuracy.py): the decision margins on primitive
pairs whose geometry is known in closed form, the per-vertex bound, and the
comparator on planted differences.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1812_04719_gb300 import accuracy as A
from paper_1812_04719_gb300 import scenegen as G


def test_vf_margins_closed_form():
    """A vertex falling through a static right triangle (legs 1 along x and y,
    in z = 0) at (0.2, 0.3): contact at tau = 1/2 with barycentrics
    (0.5, 0.2, 0.3); its distances to the three edge lines are 0.5/sqrt(2),
    0.2 and 0.3, so the inside margin is 0.2; the normal speed is 2, so the
    time margin is 1; no tangential motion.  The oracle's contact test gives
    the same tau and weights."""
    X0 = np.array([[0.2, 0.3, 1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    X1 = X0.copy()
    X1[0, 2] = -1.0
    st, tau, w1, w2 = O.ccd_primitive("vf", X0, X1)
    assert st == 1 and tau == 0.5 and abs(w1 - 0.2) < 1e-15 and abs(w2 - 0.3) < 1e-15
    ins, tm, vn, vt = A.margins(np.array([0]), X0[None], X1[None], np.array([tau]), np.array([[w1, w2]]))
    assert abs(ins[0] - 0.2) < 1e-14 and abs(tm[0] - 1.0) < 1e-14
    assert abs(vn[0] - 2.0) < 1e-14 and vt[0] < 1e-14
    # tangential motion of the vertex (0.4 in x over the step): the margin in
    # bound units shrinks by 1 + v_t / v_n = 1.2
    X1t = X1.copy()
    X1t[0, 0] += 0.4
    st, tau, w1, w2 = O.ccd_primitive("vf", X0, X1t)
    ins, tm, vn, vt = A.margins(np.array([0]), X0[None], X1t[None], np.array([tau]), np.array([[w1, w2]]))
    assert abs(vt[0] - 0.4) < 1e-14 and abs(vn[0] - 2.0) < 1e-14
    d = 1e-3
    mu = A.scaled_margin(ins, tm, vn, vt, np.array([d]))
    assert abs(mu[0] - min(ins[0] / (d * 1.2), tm[0] / d)) < 1e-9


def test_ee_margins_closed_form():
    """Edge p from (0,0,0) to (2,0,0) (static) and edge q from (0.5,-1,1) to
    (0.5,1,1) falling to z = -1: they cross at s = 1/4, u = 1/2, tau = 1/2,
    at right angles; the inside margin is min(s, 1-s)|p| = 0.5 against
    min(u, 1-u)|q| = 1, times sin 90 deg; the time margin 1/2 * 2."""
    X0 = np.array([[0, 0, 0], [2, 0, 0], [0.5, -1, 1], [0.5, 1, 1]], dtype=np.float64)
    X1 = X0.copy()
    X1[2:, 2] = -1.0
    st, tau, s, u = O.ccd_primitive("ee", X0, X1)
    assert st == 1 and tau == 0.5 and s == 0.25 and u == 0.5
    ins, tm, vn, vt = A.margins(np.array([2]), X0[None], X1[None], np.array([tau]), np.array([[s, u]]))
    assert abs(ins[0] - 0.5) < 1e-14 and abs(tm[0] - 1.0) < 1e-14 and abs(vn[0] - 2.0) < 1e-14


def test_point_delta_matches_vertex_bound():
    sc = G.scene_small((2, 1, 1), p=4, seed=3)
    X = np.concatenate([O.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)).ravel() for v in range(sc.n)])
    pd = A.point_delta(sc.p, sc.coef_of, sc.vert_off(), X)
    for v in range(sc.n):
        p = int(sc.p[v])
        nv = O.nverts(2 * p)
        o = int(sc.vert_off()[v])
        Xv = X[o:o + 6 * nv].reshape(2, 3, nv)
        a1 = np.abs(sc.coef_of(v)[:, :, 1:]).sum(-1)
        ref = (2.0 ** -23 * np.abs(Xv) + 2.0 ** -19 * a1[:, :, None] * math.sqrt((2 * p + 1) / (2 * math.pi)))
        assert np.array_equal(pd[o // 6:o // 6 + nv], ref.max(axis=(0, 1)))


def _oracle_result(sc, Xs, X1grad=True):
    boxes = np.stack([O.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = O.candidate_pairs(boxes, sc.L)
    c = O.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True)
    c0 = O.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True, grad_wrt="X0")
    r = dict(c)
    r["i"], r["j"] = pairs[:, 0], pairs[:, 1]
    r["shift"] = 9 * (pairs[:, 2] + 1) + 3 * (pairs[:, 3] + 1) + (pairs[:, 4] + 1)
    return r, c0["grad"]


@pytest.fixture(scope="module")
def pair_scene():
    sc = G.scene_pair()
    Xs = [O.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    X = np.concatenate([x.ravel() for x in Xs])
    r, g0 = _oracle_result(sc, Xs)
    assert len(r["pair"]) > 20
    return sc, Xs, X, r, g0


def test_contact_points_are_the_oracle_points(pair_scene):
    """contact_points reads each contact's four points (second vesicle at its
    image) from gves/gvid: re-running the oracle's single-pair test on them
    gives the contact's own tau and weights."""
    sc, Xs, X, r, g0 = pair_scene
    X0, X1 = A.contact_points(r, X, sc.vert_off(), sc.L)
    for k in range(len(r["pair"])):
        st, tau, w1, w2 = O.ccd_primitive("ee" if r["type"][k] == 2 else "vf", X0[k], X1[k])
        assert st == 1 and tau == r["tau"][k] and (w1, w2) == tuple(r["w"][k])


def test_compare_identical_and_planted(pair_scene):
    """Identical results satisfy every bound with zero error; a contact
    volume moved beyond S delta, a gradient row moved beyond 4 kappa, a
    robust contact dropped from one list: each is caught."""
    sc, Xs, X, r, g0 = pair_scene
    pd = A.point_delta(sc.p, sc.coef_of, sc.vert_off(), X)
    res = A.compare(r, X, r, X, g0, pd, sc.vert_off(), sc.L)
    assert res["V_ratio_max"] == 0.0 and res["grad_rel_max"] == 0.0 and res["only_mixed"] == 0
    assert res["bound1_V_holds"] and res["bound2_lists_hold"] and res["bound3_grad_holds"] and res["bound4_pairs_hold"]
    # V of one contact moved by twice its first-order bound
    k = int(np.argmax(r["V"]))
    S = np.abs(r["grad"][k]).sum() + np.abs(g0[k]).sum()
    dk = pd[sc.vert_off()[r["gves"][k]] // 6 + r["gvid"][k]].max()
    ra = dict(r)
    ra["V"] = r["V"].copy()
    ra["V"][k] += 2.0 * S * dk
    res = A.compare(ra, X, r, X, g0, pd, sc.vert_off(), sc.L)
    assert not res["bound1_V_holds"] and res["bound4_pairs_hold"]
    # a pair volume moved by twice the sum of its contacts' bounds
    ra = dict(r)
    m = r["pair"] == r["pair"][k]
    dks = pd[sc.vert_off()[r["gves"][m]] // 6 + r["gvid"][m]].max(axis=1)
    pb = ((np.abs(r["grad"][m]).reshape(m.sum(), -1).sum(1) + np.abs(g0[m]).reshape(m.sum(), -1).sum(1)) * dks).sum()
    ra["V_pair"] = r["V_pair"].copy()
    ra["V_pair"][r["pair"][k]] += 2.0 * pb
    res = A.compare(ra, X, r, X, g0, pd, sc.vert_off(), sc.L)
    assert res["bound1_V_holds"] and not res["bound4_pairs_hold"]
    # a gradient row moved by 8 kappa relative to its largest entry
    ra = dict(r)
    ra["grad"] = r["grad"].copy()
    kap = S * dk / r["V"][k]
    ra["grad"][k, 0, 0] += 8 * kap * np.abs(r["grad"][k]).max()
    assert not A.compare(ra, X, r, X, g0, pd, sc.vert_off(), sc.L)["bound3_grad_holds"]
    # the most robust contact missing from the MIXED list
    X0, X1 = A.contact_points(r, X, sc.vert_off(), sc.L)
    ins, tm, vn, vt = A.margins(r["type"], X0, X1, r["tau"], r["w"])
    dks = pd[sc.vert_off()[r["gves"]] // 6 + r["gvid"]].max(axis=1)
    mu = A.scaled_margin(ins, tm, vn, vt, dks)
    k = int(np.argmax(mu))
    assert mu[k] > A.MARGIN_FACTOR
    keep = np.arange(len(r["pair"])) != k
    ra = {key: (v[keep] if key in ("pair", "type", "a", "b", "tau", "w", "V", "grad", "gves", "gvid") else v)
          for key, v in r.items()}
    res = A.compare(ra, X, r, X, g0, pd, sc.vert_off(), sc.L)
    assert res["only_fp64"] == 1 and not res["bound2_lists_hold"]
