"""Pins of the literal-reading variants of Eq. 3.2 (U_k the absolute velocity
of the contact point) and of the gradient with respect to X0."""
import math

import numpy as np
import pytest

E_DT = 0.1   # eps * dt


def vf_moving_triangle(speed=0.8, h=0.3):
    """Static vertex at the origin; the triangle (legs 1 and 2 in the plane
    z = h) moves straight down by `speed` over the step."""
    tri0 = np.array([[-0.4, -0.3, h], [0.6, -0.3, h], [-0.4, 1.7, h]])
    X0 = np.vstack([[0.0, 0.0, 0.0], tri0])
    X1 = X0.copy()
    X1[1:, 2] -= speed
    return X0, X1


def test_vf_closed_forms(orc):
    """Triangle moving onto a static vertex: tau = h / speed; |m| = |a x b|
    = 2 (legs 1 and 2, translated rigidly); the relative reading gives
    0.5 (1-tau) |m| sqrt((eps dt)^2 + speed^2), the literal (absolute) one
    0.5 (1-tau) (eps dt) |m|, because the vertex does not move."""
    speed, h = 0.8, 0.3
    X0, X1 = vf_moving_triangle(speed, h)
    tau = h / speed
    st, V_rel, _ = orc.stiv_primitive_variant("vf", X0, X1, E_DT, "relative")
    st2, V_abs, _ = orc.stiv_primitive_variant("vf", X0, X1, E_DT, "absolute")
    assert st == st2 == 1
    assert abs(V_rel - 0.5 * (1 - tau) * 2.0 * math.sqrt(E_DT ** 2 + speed ** 2)) < 1e-14
    assert abs(V_abs - 0.5 * (1 - tau) * E_DT * 2.0) < 1e-14


def test_vf_static_triangle_readings_agree(orc):
    """Vertex moving onto a static triangle: its absolute velocity is the
    relative one, so both readings give the same V."""
    X0, X1 = vf_moving_triangle()
    # swap roles: move the vertex up by the same amount, keep the triangle still
    Y0 = X0.copy(); Y1 = X0.copy(); Y1[0, 2] += 0.8
    _, V_rel, g_rel = orc.stiv_primitive_variant("vf", Y0, Y1, E_DT, "relative")
    _, V_abs, g_abs = orc.stiv_primitive_variant("vf", Y0, Y1, E_DT, "absolute")
    assert V_rel > 0 and abs(V_rel - V_abs) < 1e-15
    # the gradients differ: only the relative reading sees the triangle's velocity
    assert np.abs(g_rel[1:] - g_abs[1:]).max() > 1e-6


def test_ee_closed_forms(orc):
    """Perpendicular edges 1.5 x 2.0 apart by h = 0.2 along z.  Edge 1 moving
    down by v onto a static edge 2: both readings give 0.5 (1-tau)
    sqrt((eps dt |m|)^2 + (v |m|)^2), |m| = 3.  Edge 2 moving up instead: the
    literal reading (velocity of the point on edge 1, at rest) gives
    0.5 (1-tau) eps dt |m|."""
    h, v = 0.2, 0.5
    p0, p1 = np.array([-0.5, 0.3, h]), np.array([1.0, 0.3, h])
    q0, q1 = np.array([0.2, -0.8, 0.0]), np.array([0.2, 1.2, 0.0])
    X0 = np.array([p0, p1, q0, q1])
    X1 = X0.copy(); X1[:2, 2] -= v
    tau = h / v
    m = 1.5 * 2.0
    ref = 0.5 * (1 - tau) * math.sqrt((E_DT * m) ** 2 + (v * m) ** 2)
    for vel in ("relative", "absolute"):
        st, V, _ = orc.stiv_primitive_variant("ee", X0, X1, E_DT, vel)
        assert st == 1 and abs(V - ref) < 1e-14, (vel, V, ref)
    X1 = X0.copy(); X1[2:, 2] += v
    _, V_rel, _ = orc.stiv_primitive_variant("ee", X0, X1, E_DT, "relative")
    _, V_abs, _ = orc.stiv_primitive_variant("ee", X0, X1, E_DT, "absolute")
    assert abs(V_rel - ref) < 1e-14
    assert abs(V_abs - 0.5 * (1 - tau) * E_DT * m) < 1e-14


def random_hits(orc, kind, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        X0 = rng.normal(size=(4, 3))
        X1 = X0 + rng.normal(scale=0.8, size=(4, 3))
        st, V, _ = orc.stiv_primitive_variant(kind, X0, X1, E_DT)
        if st == 1 and V > 1e-3:
            out.append((X0, X1))
    return out


@pytest.mark.parametrize("kind", ["vf", "ee"])
@pytest.mark.parametrize("vel", ["relative", "absolute"])
def test_grad_x0_finite_differences(orc, kind, vel):
    """dV/dX0 against central differences, h = 1e-6, on cases whose contact
    survives the perturbation."""
    h = 1e-6
    checked = 0
    for X0, X1 in random_hits(orc, kind, 12, seed=10 * ("vf", "ee").index(kind) + ("relative", "absolute").index(vel)):
        _, V, g = orc.stiv_primitive_variant(kind, X0, X1, E_DT, vel, "X0")
        ok = True
        fd = np.zeros((4, 3))
        for q in range(4):
            for c in range(3):
                Vs = []
                for sgn in (1, -1):
                    Y = X0.copy(); Y[q, c] += sgn * h
                    st, Vh, _ = orc.stiv_primitive_variant(kind, Y, X1, E_DT, vel)
                    ok = ok and st == 1
                    Vs.append(Vh)
                fd[q, c] = (Vs[0] - Vs[1]) / (2 * h)
        if not ok:
            continue
        assert np.abs(fd - g).max() <= 1e-5 * max(np.abs(g).max(), 1e-3), (fd, g)
        checked += 1
    assert checked >= 8


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_translation_identities(orc, kind):
    """A rigid translation of both time levels leaves V unchanged in both
    readings: sum_q (dV/dX0_q + dV/dX1_q) = 0.  Adding one displacement to
    every point's X1 leaves the relative reading unchanged (sum_q dV/dX1_q =
    0) but not the literal one."""
    broke = 0
    for X0, X1 in random_hits(orc, kind, 10, seed=11):
        for vel in ("relative", "absolute"):
            _, V, g1 = orc.stiv_primitive_variant(kind, X0, X1, E_DT, vel, "X1")
            _, _, g0 = orc.stiv_primitive_variant(kind, X0, X1, E_DT, vel, "X0")
            scale = max(np.abs(g1).max(), np.abs(g0).max())
            assert np.abs((g0 + g1).sum(axis=0)).max() <= 1e-10 * scale
            if vel == "relative":
                assert np.abs(g1.sum(axis=0)).max() <= 1e-10 * scale
            elif np.abs(g1.sum(axis=0)).max() > 1e-6 * scale:
                broke += 1
    assert broke >= 5


def test_scene_variants(orc):
    """On a scene: the contact lists do not depend on the reading of U_k;
    V > 0 in both readings (the eps dt |m| term); the X0 and X1 rows of
    each contact sum to zero (rigid translation)."""
    from paper_1812_04719_gb300 import scenegen as G
    sc = G.scene_small((2, 2, 1), p=4, seed=3)
    Xs = [orc.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    r = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt)
    a = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, velocity="absolute")
    g0 = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad_wrt="X0")
    assert len(r["pair"]) > 50
    for k in ("pair", "type", "a", "b", "tau", "w"):
        assert np.array_equal(r[k], a[k]) and np.array_equal(r[k], g0[k]), k
    assert np.all(a["V"] > 0) and np.any(np.abs(a["V"] - r["V"]) > 1e-6 * r["V"])
    assert np.array_equal(r["V"], g0["V"])
    s = (g0["grad"] + r["grad"]).sum(axis=1)
    assert np.abs(s).max() <= 1e-10 * np.abs(r["grad"]).max()
