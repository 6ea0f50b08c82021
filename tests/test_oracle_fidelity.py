"""Pins of the oracle's mesh-fidelity estimate (Sec. 3.1.2: the q^up-grid
triangle mesh against the smooth SH surface, ||X^{q^up} - X||_inf; Fig. 6:
a 4x upsampled grid stands in for the smooth surface)."""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

from paper_1812_04719_gb300 import scenegen as G


def real_sh_scipy(n, m, theta, phi):
    """Real orthonormal SH without Condon-Shortley phase, from scipy's complex
    Y_n^m (which carries the (-1)^m phase)."""
    am = abs(m)
    y = sph_harm_y(n, am, theta, phi) * (-1) ** am
    if m == 0:
        return y.real
    if m > 0:
        return math.sqrt(2) * y.real
    return math.sqrt(2) * y.imag


def ring_thetas(P):
    x, _ = np.polynomial.legendre.leggauss(P + 1)
    return np.arccos(x[::-1])


def shape(seed=1, p=6):
    """A perturbed prolate vesicle of order p (one time level), from the
    seeded scene generator."""
    rng = np.random.default_rng(seed)
    a, b = G.prolate_axes()
    M = G.random_rotation(rng) @ np.diag([b, b, a])
    return G.ellipsoid_coef(p, np.array([0.3, -0.2, 0.1]), M) + G.perturbation(rng, p, 0.02)


def sphere(R, center, p=2):
    coef = np.zeros((3, (p + 1) ** 2))
    coef[:, 0] = math.sqrt(4 * math.pi) * np.asarray(center)
    k = math.sqrt(4 * math.pi / 3) * R        # x = R sin cos, y = R sin sin, z = R cos
    coef[0, 3] = k      # (1, +1): cos phi
    coef[1, 1] = k      # (1, -1): sin phi
    coef[2, 2] = k      # (1, 0)
    return coef


def test_sphere_coefficients(orc):
    """The sphere's series synthesises points at distance R from the centre."""
    P = 8
    X = orc.synth_vesicle(2, P, np.stack([sphere(1.3, [0.2, 0.1, -0.4])] * 2))[0]
    r = np.linalg.norm(X - np.array([0.2, 0.1, -0.4])[:, None], axis=0)
    assert np.abs(r - 1.3).max() < 1e-14


@pytest.mark.parametrize("P", [4, 8])
def test_mesh_point_at_vertices(orc, P):
    """At every grid vertex (theta_i, phi_j) the mesh is the vertex itself."""
    coef = shape()
    p = 6
    X = orc.synth_vesicle(p, P, np.stack([coef, coef]))[0]
    th = ring_thetas(P)
    for i in range(P + 1):
        for j in range(2 * P):
            got = orc.mesh_point(P, X, th[i], math.pi * j / P)
            assert np.abs(got - X[:, i * 2 * P + j]).max() <= 1e-14 * np.abs(X).max()


def test_mesh_point_on_mesh_triangles(orc):
    """Every mesh point lies on a triangle of the mesh's own triangle list
    (the Fig. 3 split and pole fans), one whose corners are the grid cell's;
    the other diagonal's triangles are not in that list."""
    P, p = 6, 6
    coef = shape(seed=3)
    X = orc.synth_vesicle(p, P, np.stack([coef, coef]))[0]
    tris = orc.triangles(P)
    rng = np.random.default_rng(0)
    for _ in range(300):
        theta, phi = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
        y = orc.mesh_point(P, X, theta, phi)
        best = np.inf
        for t in tris:
            A, B, C = X[:, t[0]], X[:, t[1]], X[:, t[2]]
            e1, e2, d = B - A, C - A, y - A
            M = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
            u, v = np.linalg.solve(M, [d @ e1, d @ e2])
            if u >= -1e-9 and v >= -1e-9 and u + v <= 1 + 1e-9:
                best = min(best, np.linalg.norm(A + u * e1 + v * e2 - y))
        assert best < 1e-12, (theta, phi, best)


def test_mesh_point_continuous(orc):
    """The map is continuous across ring boundaries, cell boundaries in phi
    and the split diagonal."""
    P, p = 8, 6
    coef = shape(seed=5)
    X = orc.synth_vesicle(p, P, np.stack([coef, coef]))[0]
    th = ring_thetas(P)
    h = 1e-11
    for i in range(P + 1):
        for phi in (0.3, 1.7, 4.4):
            a, b = orc.mesh_point(P, X, th[i] - h, phi), orc.mesh_point(P, X, th[i] + h, phi)
            assert np.abs(a - b).max() < 1e-8
    for j in range(2 * P):
        for theta in (0.05, 1.0, 2.2, 3.1):
            pj = math.pi * j / P
            a, b = orc.mesh_point(P, X, theta, pj - h), orc.mesh_point(P, X, theta, pj + h)
            assert np.abs(a - b).max() < 1e-8
    # along the diagonal (i, j)-(i+1, j+1) of a cell both triangles agree
    i, j = 3, 5
    for s_ in (0.2, 0.5, 0.8):
        theta = th[i] + s_ * (th[i + 1] - th[i])
        phi = math.pi * (j + s_) / P
        a, b = orc.mesh_point(P, X, theta + h, phi), orc.mesh_point(P, X, theta - h, phi)
        assert np.abs(a - b).max() < 1e-8


def test_sphere_meridian_chord(orc):
    """On a sphere, a mesh point on a grid meridian between rings i and i+1
    (fraction a) is on the chord: its distance from the centre is
    R sqrt((1-a)^2 + a^2 + 2 a (1-a) cos(theta_{i+1} - theta_i))."""
    P, R, c = 8, 1.3, np.array([0.2, 0.1, -0.4])
    X = orc.synth_vesicle(2, P, np.stack([sphere(R, c)] * 2))[0]
    th = ring_thetas(P)
    for i in range(P):
        for a in (0.25, 0.5, 0.9):
            theta = th[i] + a * (th[i + 1] - th[i])
            y = orc.mesh_point(P, X, theta, math.pi * 3 / P)
            D = th[i + 1] - th[i]
            ref = R * math.sqrt((1 - a) ** 2 + a * a + 2 * a * (1 - a) * math.cos(D))
            assert abs(np.linalg.norm(y - c) - ref) < 1e-13


def test_fidelity_brute_force(orc):
    """The estimate is the largest distance over the order-(factor P) grid,
    recomputed here with scipy's spherical harmonics for the smooth surface."""
    p, P, factor = 4, 4, 2
    coef = shape(seed=7, p=p)
    X = orc.synth_vesicle(p, P, np.stack([coef, coef]))[0]
    Pf = factor * P
    worst = 0.0
    for theta in ring_thetas(Pf):
        for k in range(2 * Pf):
            phi = math.pi * k / Pf
            smooth = np.zeros(3)
            for n in range(p + 1):
                for m in range(-n, n + 1):
                    smooth += coef[:, n * n + n + m] * real_sh_scipy(n, m, theta, phi)
            worst = max(worst, float(np.linalg.norm(orc.mesh_point(P, X, theta, phi) - smooth)))
    assert abs(orc.mesh_fidelity(p, P, coef, X, factor) - worst) <= 1e-13 * worst


def test_fidelity_second_order(orc):
    """Linear interpolation: the error falls by about 4 when P doubles."""
    p = 6
    coef = shape(seed=2, p=p)
    e = [orc.mesh_fidelity(p, P, coef, orc.synth_vesicle(p, P, np.stack([coef, coef]))[0]) for P in (16, 32, 64)]
    assert 3.3 < e[0] / e[1] < 4.5 and 3.6 < e[1] / e[2] < 4.4, e


def test_fidelity_translation_and_scale(orc):
    """A rigid translation leaves the error unchanged; scaling the surface
    scales it."""
    p, P = 6, 12
    coef = shape(seed=4, p=p)
    e0 = orc.mesh_fidelity(p, P, coef, orc.synth_vesicle(p, P, np.stack([coef, coef]))[0])
    moved = coef.copy()
    moved[:, 0] += math.sqrt(4 * math.pi) * np.array([5.0, -3.0, 2.0])
    e1 = orc.mesh_fidelity(p, P, moved, orc.synth_vesicle(p, P, np.stack([moved, moved]))[0])
    scaled = 2.5 * coef
    e2 = orc.mesh_fidelity(p, P, scaled, orc.synth_vesicle(p, P, np.stack([scaled, scaled]))[0])
    assert abs(e1 - e0) <= 1e-12 * e0 + 1e-14
    assert abs(e2 - 2.5 * e0) <= 1e-12 * e0
