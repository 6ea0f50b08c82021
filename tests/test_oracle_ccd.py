"""Pins of the oracle's contact time (Eq. 3.1 with d_m = 0) and inside tests,
against closed forms and exact rational arithmetic."""
from fractions import Fraction as Fr

import numpy as np
import pytest


def exact_poly(kind, X0, X1):
    """Exact coefficients of the coplanarity cubic from 4 exact samples
    (independent of the oracle's coefficient formulas)."""
    X0 = [[Fr(float(v)) for v in r] for r in np.asarray(X0).reshape(4, 3)]
    X1 = [[Fr(float(v)) for v in r] for r in np.asarray(X1).reshape(4, 3)]

    def pos(q, t):
        return [X0[q][c] + t * (X1[q][c] - X0[q][c]) for c in range(3)]

    def sub(u, v):
        return [u[c] - v[c] for c in range(3)]

    def cross(u, v):
        return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]

    def dot(u, v):
        return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]

    def f(t):
        Y = [pos(q, t) for q in range(4)]
        if kind == "vf":
            return dot(sub(Y[0], Y[1]), cross(sub(Y[2], Y[1]), sub(Y[3], Y[1])))
        return dot(sub(Y[2], Y[0]), cross(sub(Y[1], Y[0]), sub(Y[3], Y[2])))

    ts = [Fr(0), Fr(1, 3), Fr(2, 3), Fr(1)]
    fs = [f(t) for t in ts]
    # Newton divided differences -> monomial coefficients
    A = [[t ** k for k in range(4)] for t in ts]
    # solve 4x4 exactly (Gauss)
    M = [row[:] + [fv] for row, fv in zip(A, fs)]
    for i in range(4):
        piv = next(r for r in range(i, 4) if M[r][i] != 0)
        M[i], M[piv] = M[piv], M[i]
        for r in range(4):
            if r != i and M[r][i] != 0:
                fac = M[r][i] / M[i][i]
                M[r] = [M[r][k] - fac * M[i][k] for k in range(5)]
    k = [M[i][4] / M[i][i] for i in range(4)]
    return k, pos, f


def exact_inside(kind, Y):
    def sub(u, v):
        return [u[c] - v[c] for c in range(3)]

    def dot(u, v):
        return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]
    if kind == "vf":
        a, b, c = sub(Y[2], Y[1]), sub(Y[3], Y[1]), sub(Y[0], Y[1])
        d00, d01, d11, d20, d21 = dot(a, a), dot(a, b), dot(b, b), dot(c, a), dot(c, b)
        den = d00 * d11 - d01 * d01
        b1 = (d11 * d20 - d01 * d21) / den
        b2 = (d00 * d21 - d01 * d20) / den
        return (b1, b2), min(1 - b1 - b2, b1, b2)
    d1, d2, r = sub(Y[1], Y[0]), sub(Y[3], Y[2]), sub(Y[0], Y[2])
    A, B, E, C, F = dot(d1, d1), dot(d1, d2), dot(d2, d2), dot(d1, r), dot(d2, r)
    den = A * E - B * B
    s = (B * F - C * E) / den
    u = (A * F - B * C) / den
    return (s, u), min(s, 1 - s, u, 1 - u)


def exact_ccd(kind, X0, X1):
    """Earliest root in [0,1] (exact bisection to 2^-80) whose point passes the
    exact inside test.  Returns (hit, tau, weights, margin)."""
    k, pos, f = exact_poly(kind, X0, X1)

    def fv(t):
        return ((k[3] * t + k[2]) * t + k[1]) * t + k[0]
    grid = [Fr(i, 512) for i in range(513)]
    roots = []
    for lo, hi in zip(grid[:-1], grid[1:]):
        flo, fhi = fv(lo), fv(hi)
        if flo == 0:
            roots.append(lo)
            continue
        if (flo < 0) != (fhi < 0) and fhi != 0:
            for _ in range(80):
                mid = (lo + hi) / 2
                if (fv(mid) < 0) == (flo < 0):
                    lo = mid
                else:
                    hi = mid
            roots.append(lo)
    if fv(Fr(1)) == 0:
        roots.append(Fr(1))
    for t in roots:
        Y = [pos(q, t) for q in range(4)]
        w, margin = exact_inside(kind, Y)
        if margin >= 0:
            return True, t, w, margin
    return False, None, None, None


def test_vf_closed_form_rational(orc):
    X0 = np.array([[0.25, 0.25, 1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]])
    X1 = np.array([[0.25, 0.25, -1.0], [0, 0, 0], [1, 0, 0], [0, 1, 0]])
    st, tau, b1, b2 = orc.ccd_primitive("vf", X0, X1)
    assert st == 1 and tau == 0.5 and b1 == 0.25 and b2 == 0.25


def test_vf_vertex_toward_static_triangle(orc):
    """tau = d0 / (D . n_hat) for a vertex moving at constant speed."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        tri = rng.normal(size=(3, 3))
        n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        n /= np.linalg.norm(n)
        bary = rng.dirichlet([2, 2, 2])
        hit = bary @ tri
        d0 = rng.uniform(0.1, 1.0)
        D = -n * d0 / rng.uniform(0.2, 0.8) + np.cross(n, rng.normal(size=3)) * 0.1
        xp0 = hit + n * d0 - (D - (D @ n) * n) * 0  # start above the plane
        xp0 = xp0 - (D - (D @ n) * n) * (d0 / -(D @ n))
        X0 = np.vstack([xp0, tri])
        X1 = np.vstack([xp0 + D, tri])
        st, tau, b1, b2 = orc.ccd_primitive("vf", X0, X1)
        tau_ref = d0 / -(D @ n)
        assert st == 1
        assert abs(tau - tau_ref) < 1e-13
        assert abs(b1 - bary[1]) < 1e-11 and abs(b2 - bary[2]) < 1e-11


def test_ee_perpendicular_crossing(orc):
    X0 = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0.5], [0, 1, 0.5]], dtype=float)
    X1 = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -0.5], [0, 1, -0.5]], dtype=float)
    st, tau, s, u = orc.ccd_primitive("ee", X0, X1)
    assert st == 1 and tau == 0.5 and s == 0.5 and u == 0.5
    # offset the moving edge beyond the end of the static one: lines cross, edges do not
    X0[2:, 0] += 1.5
    X1[2:, 0] += 1.5
    assert orc.ccd_primitive("ee", X0, X1)[0] == 0


def test_grazing_miss_and_parallel_motion(orc):
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    # crosses the plane outside the triangle
    X0 = np.vstack([[0.8, 0.8, 1.0], tri]); X1 = np.vstack([[0.8, 0.8, -1.0], tri])
    assert orc.ccd_primitive("vf", X0, X1)[0] == 0
    # moves parallel to the plane
    X0 = np.vstack([[0.2, 0.2, 0.1], tri]); X1 = np.vstack([[0.3, 0.1, 0.1], tri])
    assert orc.ccd_primitive("vf", X0, X1)[0] == 0


def test_tie_on_triangle_edge_counts(orc):
    """A vertex crossing exactly on an edge (beta = 0 exactly) is a contact:
    the triangle is closed."""
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    X0 = np.vstack([[0.5, 0.0, 1.0], tri]); X1 = np.vstack([[0.5, 0.0, -1.0], tri])
    st, tau, b1, b2 = orc.ccd_primitive("vf", X0, X1)
    assert st == 1 and tau == 0.5 and b2 == 0.0
    # just outside the edge
    X0[0, 1] = X1[0, 1] = -2.0 ** -40
    assert orc.ccd_primitive("vf", X0, X1)[0] == 0


def test_coplanar_throughout_is_degenerate(orc):
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    X0 = np.vstack([[0.2, 0.2, 0.0], tri]); X1 = np.vstack([[0.3, 0.1, 0.0], tri])
    assert orc.ccd_primitive("vf", X0, X1)[0] == 2


def test_start_in_contact(orc):
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    X0 = np.vstack([[0.2, 0.2, 0.0], tri]); X1 = np.vstack([[0.2, 0.2, -0.5], tri])
    st, tau, _, _ = orc.ccd_primitive("vf", X0, X1)
    assert st == 1 and tau == 0.0


@pytest.mark.parametrize("kind", ["vf", "ee"])
def test_random_against_exact_rationals(orc, kind):
    """Random crossing configurations: contact decision, earliest tau and weights
    against exact rational arithmetic (exact cubic from 4 samples, exact
    bisection, exact inside test).  Cases within 1e-9 of a decision boundary
    are skipped."""
    rng = np.random.default_rng(42 if kind == "vf" else 43)
    checked = hits = 0
    for _ in range(250):
        X0 = rng.normal(size=(4, 3)) * np.array([1.0, 1.0, 0.2])
        X1 = X0 + rng.normal(size=(4, 3)) * 0.3
        if kind == "vf":
            X0[0] = X0[1:].mean(0) + rng.normal(size=3) * 0.4
            X1[0] = X1[1:].mean(0) + rng.normal(size=3) * 0.4
            X0[0, 2] += 1.0; X1[0, 2] -= 1.0
        else:
            X0[2:, 2] += 1.0; X1[2:, 2] -= 1.0
        hit, tau, w, margin = exact_ccd(kind, X0, X1)
        if hit and margin < 1e-9:
            continue
        st, t, w1, w2 = orc.ccd_primitive(kind, X0, X1)
        if st == 2:
            continue
        checked += 1
        assert (st == 1) == hit
        if hit:
            hits += 1
            assert abs(t - float(tau)) < 1e-13
            assert abs(w1 - float(w[0])) < 1e-9 and abs(w2 - float(w[1])) < 1e-9
    assert checked > 200 and hits > 20
