"""Pins of the oracle's SH synthesis (Sec. 3.1.1, Sec. 3.1.2 upsampling)
against library routines, closed forms and quadrature identities."""
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


def grid_angles_numpy(P):
    x, _ = np.polynomial.legendre.leggauss(P + 1)
    theta = np.arccos(x[::-1])  # ascending theta
    phi = 2 * np.pi * np.arange(2 * P) / (2 * P)
    th = np.concatenate([np.repeat(theta, 2 * P), [0.0, np.pi]])
    ph = np.concatenate([np.tile(phi, P + 1), [0.0, 0.0]])
    return th, ph


@pytest.mark.parametrize("nq", [2, 5, 17, 25, 33, 65])
def test_gl_nodes_match_numpy(orc, nq):
    x, w = orc.gl_nodes(nq)
    xr, wr = np.polynomial.legendre.leggauss(nq)
    assert np.all(np.diff(x) < 0), "nodes must be sorted so that theta ascends"
    assert np.abs(x[::-1] - xr).max() < 1e-15
    assert np.abs(w[::-1] - wr).max() < 2e-15


@pytest.mark.parametrize("nmax", [4, 16, 32])
def test_legendre_matches_scipy(orc, nmax):
    rng = np.random.default_rng(nmax)
    for th in rng.uniform(0, np.pi, 7):
        P = orc.legendre_norm(nmax, math.cos(th))
        for n in range(nmax + 1):
            for m in range(n + 1):
                ref = sph_harm_y(n, m, th, 0.0).real * (-1) ** m
                assert abs(P[n * (n + 1) // 2 + m] - ref) < 5e-14 * max(1.0, abs(ref))


@pytest.mark.parametrize("p", [2, 4, 8, 12])
def test_synthesis_matches_scipy_basis(orc, p):
    P = 2 * p
    rng = np.random.default_rng(p)
    coef = rng.normal(size=(p + 1) ** 2) / np.repeat(np.arange(1, p + 2) ** 2, 2 * np.arange(p + 1) + 1)
    th, ph = grid_angles_numpy(P)
    ref = np.zeros_like(th)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            ref += coef[n * n + n + m] * real_sh_scipy(n, m, th, ph)
    got = orc.synth(p, P, coef)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(coef).sum()


def test_ellipsoid_closed_form(orc):
    """An ellipsoid c + M u is exactly degree 1: grid points equal the closed form."""
    rng = np.random.default_rng(3)
    a, b = G.prolate_axes()
    for p in (1, 4, 8, 16):
        P = 2 * p
        R = G.random_rotation(rng)
        M = R @ np.diag([b, b, a])
        c = rng.uniform(-20, 20, 3)
        coef = G.ellipsoid_coef(p, c, M)
        th, ph = grid_angles_numpy(P)
        u = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        ref = c[:, None] + M @ u
        got = np.stack([orc.synth(p, P, coef[k]) for k in range(3)])
        assert np.abs(got - ref).max() < 1e-13


def test_prolate_shape_matches_paper():
    """Reduced volume 0.91 at R0 = 1.34 (Sec. 4.3): semi-axes and volume."""
    a, b = G.prolate_axes()
    assert abs(a / b - 1.8864) < 2e-4
    assert abs(a - 1.9825) < 1e-4 and abs(b - 1.0509) < 1e-4
    assert abs(4.0 / 3.0 * math.pi * a * b * b - 9.1716) < 1e-3


@pytest.mark.parametrize("p", [3, 8])
def test_quadrature_round_trip(orc, p):
    """Gauss-Legendre x trapezoidal analysis of the synthesized grid returns the
    coefficients (exact for products of degree <= 2p on the 2p grid)."""
    P = 2 * p
    rng = np.random.default_rng(11 + p)
    coef = rng.normal(size=(p + 1) ** 2)
    vals = orc.synth(p, P, coef)[: 2 * P * (P + 1)].reshape(P + 1, 2 * P)
    x, w = np.polynomial.legendre.leggauss(P + 1)
    theta, wq = np.arccos(x[::-1]), w[::-1]
    phi = 2 * np.pi * np.arange(2 * P) / (2 * P)
    got = np.zeros_like(coef)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            Y = real_sh_scipy(n, m, theta[:, None], phi[None, :])
            got[n * n + n + m] = np.sum(wq[:, None] * (np.pi / P) * vals * Y)
    assert np.abs(got - coef).max() < 1e-12


def test_adjoint_is_transpose(orc):
    """S^T g equals the transpose of the dense synthesis matrix built from scipy."""
    p, P = 4, 8
    th, ph = grid_angles_numpy(P)
    S = np.stack([real_sh_scipy(n, m, th, ph) for n in range(p + 1) for m in range(-n, n + 1)], axis=1)
    rng = np.random.default_rng(5)
    g = rng.normal(size=S.shape[0])
    assert np.abs(orc.synth_adjoint(p, P, g) - S.T @ g).max() < 1e-12
