"""Pins of the oracle's contact test with minimum separation d_m > 0 (Eq. 3.1:
the degree-six equation f^2 - d_m^2 |m|^2 = 0, f the coplanarity cubic, m the
normal), its root isolation and its volume gradient."""
import numpy as np
import pytest

E_DT = 0.1


@pytest.mark.parametrize("seed", range(6))
def test_root_isolation_against_numpy(orc, seed):
    """Polynomials of degree 1-6 built from known roots (some in (0, 1), some
    outside, well separated): the isolated roots equal numpy's within 1e-12."""
    rng = np.random.default_rng(seed)
    for n in range(1, 7):
        for _ in range(20):
            while True:
                r = np.sort(rng.uniform(-0.5, 1.5, n))
                if np.min(np.diff(np.concatenate([[-9], r, [9]]))) > 0.02 and \
                        np.min(np.abs(r)) > 0.02 and np.min(np.abs(r - 1)) > 0.02:
                    break
            c = np.polynomial.polynomial.polyfromroots(r) * rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 3.0)
            got = orc.poly_roots01(c)
            ref = r[(r > 0) & (r < 1)]
            assert len(got) == len(ref), (c, got, ref)
            assert np.allclose(got, ref, atol=1e-12)


def test_multiple_roots(orc):
    """A crossing triple root in (0, 1) is found (its derivative touches zero
    there); a touching double root is not a sign change and is not reported
    (a grazing tangency is not a crossing, as in the cubic test); a
    polynomial that stays positive has no root."""
    got = orc.poly_roots01(np.polynomial.polynomial.polyfromroots([0.3, 0.3, 0.3, 2.0]))
    assert len(got) == 1 and abs(got[0] - 0.3) < 1e-4
    assert len(orc.poly_roots01(np.polynomial.polynomial.polyfromroots([0.3, 0.3, 2.0]))) == 0
    assert len(orc.poly_roots01([1.0, 0.0, 1.0])) == 0


def vf_normal_approach(h, v, d):
    """Vertex rising along the normal of a static triangle in z = 0, from
    height -h... reaching the plane's d-band at t = (h - d) / v."""
    tri = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    X0 = np.vstack([[0.1, 0.2, h], tri])
    X1 = X0.copy(); X1[0, 2] = h - v
    return X0, X1


@pytest.mark.parametrize("d", [0.01, 0.05, 0.2])
def test_vf_closed_form(orc, d):
    h, v = 0.7, 1.2
    X0, X1 = vf_normal_approach(h, v, d)
    st, tau, w1, w2 = orc.ccd_primitive_dm("vf", X0, X1, d)
    assert st == 1 and abs(tau - (h - d) / v) < 1e-14
    st0, tau0, _, _ = orc.ccd_primitive_dm("vf", X0, X1, 0.0)
    assert st0 == 1 and abs(tau0 - h / v) < 1e-15 and tau < tau0


@pytest.mark.parametrize("d", [0.01, 0.1])
def test_ee_closed_form(orc, d):
    """Perpendicular edges closing along z: the lines come within d at
    t = (h - d) / v."""
    h, v = 0.5, 0.9
    X0 = np.array([[-1.0, 0.2, h], [1.0, 0.2, h], [0.1, -1.0, 0.0], [0.1, 1.0, 0.0]])
    X1 = X0.copy(); X1[:2, 2] -= v
    st, tau, s, u = orc.ccd_primitive_dm("ee", X0, X1, d)
    assert st == 1 and abs(tau - (h - d) / v) < 1e-14
    assert abs(s - 0.55) < 1e-12 and abs(u - 0.6) < 1e-12


def test_within_band_at_start(orc):
    """Already within d_m of the plane at t = 0, above the triangle: contact at
    tau = 0; a separating vertex that never comes within d_m: none; one that
    comes within d_m only outside the triangle: none."""
    d = 0.1
    X0, X1 = vf_normal_approach(0.05, -0.5, d)   # moving away, starts inside the band
    st, tau, _, _ = orc.ccd_primitive_dm("vf", X0, X1, d)
    assert st == 1 and tau == 0.0
    X0, X1 = vf_normal_approach(0.5, 0.3, d)     # stops at 0.2 > d
    assert orc.ccd_primitive_dm("vf", X0, X1, d)[0] == 0
    X0, X1 = vf_normal_approach(0.5, 0.45, d)
    X0[0, :2] = X1[0, :2] = [5.0, 5.0]           # projection far outside the triangle
    assert orc.ccd_primitive_dm("vf", X0, X1, d)[0] == 0


def random_hits(orc, kind, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        X0 = rng.normal(size=(4, 3))
        X1 = X0 + rng.normal(scale=0.8, size=(4, 3))
        st, tau, w1, w2 = orc.ccd_primitive_dm(kind, X0, X1, 0.0)
        # keep contacts well inside the primitive, so a small band keeps them
        margin = min(w1, w2, 1 - w1 - w2) if kind == "vf" else min(w1, w2, 1 - w1, 1 - w2)
        if st == 1 and margin > 0.05 and 0.05 < tau < 0.95:
            out.append((X0, X1, tau))
    return out


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_limit_d_to_zero(orc, kind):
    """As d_m -> 0 the contact time approaches the cubic's from below, at a
    rate proportional to d_m."""
    for X0, X1, tau0 in random_hits(orc, kind, 10, seed=3):
        prev = None
        for d in (1e-3, 1e-4, 1e-5, 1e-6):
            st, tau, _, _ = orc.ccd_primitive_dm(kind, X0, X1, d)
            assert st == 1 and tau <= tau0
            gap = tau0 - tau
            if prev is not None:
                assert 5.0 < prev / gap < 20.0, (prev, gap)
            prev = gap


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_gradient_finite_differences(orc, kind):
    """dV/dX1 with tau following the degree-six equation, against central
    differences (h = 1e-6)."""
    d, h = 0.02, 1e-6
    checked = 0
    for X0, X1, _ in random_hits(orc, kind, 10, seed=5):
        st, V, g = orc.stiv_primitive_variant(kind, X0, X1, E_DT, d_m=d)
        assert st == 1 and V > 0
        fd = np.zeros((4, 3))
        ok = True
        for q in range(4):
            for c in range(3):
                vals = []
                for sgn in (1, -1):
                    Y = X1.copy(); Y[q, c] += sgn * h
                    s2, Vh, _ = orc.stiv_primitive_variant(kind, X0, Y, E_DT, d_m=d)
                    ok = ok and s2 == 1
                    vals.append(Vh)
                fd[q, c] = (vals[0] - vals[1]) / (2 * h)
        if ok:
            assert np.abs(fd - g).max() <= 1e-5 * max(np.abs(g).max(), 1e-3)
            checked += 1
    assert checked >= 8


def test_scene_band_contacts(orc):
    """On a scene with d_m > 0: at every contact time tau > 0 the point is d_m
    from the triangle's plane (the lines are d_m apart), to rounding; the
    contact test of d_m = 0 finds a subset of the primitive pairs (the band
    is reached first, so most contacts keep their keys at an earlier time);
    more primitive pairs are tested (widened boxes)."""
    from paper_1812_04719_gb300 import scenegen as G
    sc = G.scene_small((2, 2, 1), p=4, seed=3)
    Xs = [orc.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    d = 0.02
    boxes = np.stack([orc.vesicle_box(X, d) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    c0 = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt)
    cd = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, d_m=d)
    assert len(cd["pair"]) > len(c0["pair"]) > 50
    assert cd["counts"][1] > c0["counts"][1]
    L = np.broadcast_to(np.asarray(sc.L, dtype=np.float64), (3,))
    checked = 0
    for k in range(len(cd["pair"])):
        t = cd["tau"][k]
        if t == 0.0:
            continue
        row = pairs[cd["pair"][k]]
        Y = []
        for q in range(4):
            v, vid = cd["gves"][k, q], cd["gvid"][k, q]
            sh = row[2:5] * L if (v == row[1] and v != row[0]) else 0.0
            x0 = Xs[v][0][:, vid] + sh
            x1 = Xs[v][1][:, vid] + sh
            Y.append(x0 + t * (x1 - x0))
        Y = np.array(Y)
        if cd["type"][k] < 2:
            m = np.cross(Y[2] - Y[1], Y[3] - Y[1]); dist = abs((Y[0] - Y[1]) @ m) / np.linalg.norm(m)
        else:
            m = np.cross(Y[1] - Y[0], Y[3] - Y[2]); dist = abs((Y[2] - Y[0]) @ m) / np.linalg.norm(m)
        assert abs(dist - d) <= 1e-9, (k, dist)
        checked += 1
    assert checked > 50
    key = lambda c: (c["pair"].astype(np.int64) << 40) | (c["type"].astype(np.int64) << 36) | \
        (c["a"].astype(np.int64) << 18) | c["b"]
    common, i0, idd = np.intersect1d(key(c0), key(cd), return_indices=True)
    assert len(common) >= 0.9 * len(c0["pair"])
    assert np.mean(cd["tau"][idd] <= c0["tau"][i0]) > 0.8
