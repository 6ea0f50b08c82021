"""Pins of the oracle's contact volume (Eq. 3.2, App. A) and its gradient."""
import math

import numpy as np
import pytest

EPS_DT = 0.1  # eps = 1, dt = 0.1


def paper_volume(tau, dt, eps, U_rel, tri_t):
    """Eq. 3.2 as printed: (t - tau_I) sqrt(eps^2 + (U.n)^2) |t| with t - tau_I
    = (1 - tau) dt, n the unit normal and |t| the area of the triangle at tau."""
    a, b = tri_t[1] - tri_t[0], tri_t[2] - tri_t[0]
    m = np.cross(a, b)
    n = m / np.linalg.norm(m)
    return (1 - tau) * dt * math.sqrt(eps ** 2 + float(U_rel @ n) ** 2) * 0.5 * np.linalg.norm(m)


def test_vf_volume_rational(orc):
    X0 = np.array([[0.25, 0.25, 1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]])
    X1 = np.array([[0.25, 0.25, -1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]])
    st, V, g = orc.stiv_primitive("vf", X0, X1, EPS_DT)
    assert st == 1
    ref = paper_volume(0.5, 0.1, 1.0, np.array([0, 0, -2.0]) / 0.1, X0[1:])
    assert abs(V - ref) < 1e-15 * ref
    assert abs(V - 0.25 * math.sqrt(4.01)) < 1e-15


def test_vf_volume_static_triangle_random(orc):
    rng = np.random.default_rng(7)
    n_ok = 0
    for _ in range(100):
        tri = rng.normal(size=(3, 3))
        bary = rng.dirichlet([3, 3, 3])
        D = rng.normal(size=3)
        nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        if abs(D @ nrm) < 0.3 * np.linalg.norm(D) * np.linalg.norm(nrm):
            continue
        tau = rng.uniform(0.05, 0.95)
        hit = bary @ tri
        xp0 = hit - tau * D
        X0 = np.vstack([xp0, tri]); X1 = np.vstack([xp0 + D, tri])
        st, V, _ = orc.stiv_primitive("vf", X0, X1, EPS_DT)
        assert st == 1
        ref = paper_volume(tau, 0.1, 1.0, D / 0.1, tri)
        assert abs(V - ref) < 1e-11 * ref
        n_ok += 1
    assert n_ok > 50


def test_ee_volume_rational(orc):
    X0 = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0.5], [0, 1, 0.5]], dtype=float)
    X1 = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -0.5], [0, 1, -0.5]], dtype=float)
    st, V, _ = orc.stiv_primitive("ee", X0, X1, EPS_DT)
    assert st == 1
    # m = d1 x d2 = (2,0,0) x (0,2,0) = (0,0,4); D_rel = (0,0,-1)
    assert abs(V - 0.5 * 0.5 * math.sqrt(0.01 * 16 + 16)) < 1e-15


def crossing_case(rng, kind):
    while True:
        X0 = rng.normal(size=(4, 3)) * np.array([1.0, 1.0, 0.2])
        X1 = X0 + rng.normal(size=(4, 3)) * 0.3
        if kind == "vf":
            X0[0] = X0[1:].mean(0) + rng.normal(size=3) * 0.3
            X1[0] = X1[1:].mean(0) + rng.normal(size=3) * 0.3
            X0[0, 2] += 1.0; X1[0, 2] -= 1.0
        else:
            X0[2:, 2] += 1.0; X1[2:, 2] -= 1.0
        return X0, X1


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_galilean_invariance(orc, kind):
    """Adding one common displacement to all four points leaves V unchanged:
    V uses the velocity relative to the opposite primitive."""
    rng = np.random.default_rng(3)
    n = 0
    for _ in range(200):
        X0, X1 = crossing_case(rng, kind)
        st, V, _ = orc.stiv_primitive(kind, X0, X1, EPS_DT)
        if st != 1:
            continue
        w = rng.normal(size=3) * 0.5
        # moving frame: positions at time t shift by t w, so X1 shifts by w
        st2, V2, _ = orc.stiv_primitive(kind, X0, X1 + w, EPS_DT)
        if st2 != 1:
            continue
        assert abs(V2 - V) < 1e-10 * V
        n += 1
    assert n > 10


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_rigid_invariance_and_gradient_covariance(orc, kind):
    rng = np.random.default_rng(4)
    from paper_1812_04719_gb300.scenegen import random_rotation
    n = 0
    for _ in range(200):
        X0, X1 = crossing_case(rng, kind)
        st, V, g = orc.stiv_primitive(kind, X0, X1, EPS_DT)
        if st != 1:
            continue
        R = random_rotation(rng)
        t = rng.normal(size=3) * 5
        st2, V2, g2 = orc.stiv_primitive(kind, X0 @ R.T + t, X1 @ R.T + t, EPS_DT)
        if st2 != 1:
            continue
        assert abs(V2 - V) < 1e-10 * V
        assert np.abs(g2 - g @ R.T).max() < 1e-8 * np.abs(g).max()
        n += 1
    assert n > 10


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_gradient_central_differences(orc, kind):
    """dV/dX1 against central differences, h = 1e-6, where the contact
    persists at +-h."""
    rng = np.random.default_rng(5)
    h = 1e-6
    n = 0
    for _ in range(200):
        X0, X1 = crossing_case(rng, kind)
        st, V, g = orc.stiv_primitive(kind, X0, X1, EPS_DT)
        if st != 1 or V < 1e-3:
            continue
        fd = np.zeros((4, 3))
        ok = True
        for q in range(4):
            for c in range(3):
                Xp = X1.copy(); Xp[q, c] += h
                Xm = X1.copy(); Xm[q, c] -= h
                sp, Vp, _ = orc.stiv_primitive(kind, X0, Xp, EPS_DT)
                sm, Vm, _ = orc.stiv_primitive(kind, X0, Xm, EPS_DT)
                if sp != 1 or sm != 1:
                    ok = False
                fd[q, c] = (Vp - Vm) / (2 * h)
        if not ok:
            continue
        assert np.abs(fd - g).max() < 1e-6 * max(1.0, np.abs(g).max())
        n += 1
    assert n > 10


def test_volume_sign(orc):
    rng = np.random.default_rng(6)
    for _ in range(100):
        X0, X1 = crossing_case(rng, "vf")
        st, V, _ = orc.stiv_primitive("vf", X0, X1, EPS_DT)
        if st == 1:
            assert V >= 0
        else:
            assert V == 0
