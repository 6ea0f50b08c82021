"""Pins of the oracle's contact LCP (Eq. 3.7, Alg. 3, min-map Newton)."""
import numpy as np
import pytest

from oracle import lcp as L
from paper_1812_04719_gb300 import scenegen as G


def test_scalar_closed_form():
    x, it, res = L.minmap_newton(np.array([[2.5]]), np.array([-3.0]))
    assert abs(x[0] - 1.2) < 1e-15 and res < 1e-15
    x, _, _ = L.minmap_newton(np.array([[2.5]]), np.array([3.0]))
    assert x[0] == 0.0


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_newton_equals_brute_force(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        Gm = rng.normal(size=(n, n))
        B = Gm @ Gm.T + 0.1 * np.eye(n)        # positive definite: a unique solution
        q = rng.normal(size=n)
        sols = L.brute_force_lcp(B, q)
        assert len(sols) == 1
        x, _, res = L.minmap_newton(B, q)
        assert res < 1e-10
        assert np.allclose(x, sols[0], rtol=1e-9, atol=1e-12)


def _scene_lcp(orc, sc):
    Xs = [orc.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)) for v in range(sc.n)]
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True)
    hit = np.nonzero(c["V_pair"] > 0)[0]
    row_of_pair = -np.ones(len(pairs), dtype=int)
    row_of_pair[hit] = np.arange(len(hit))
    nverts = [G.nverts(int(P)) for P in sc.P]
    rows = L.jacobian_rows(len(hit), row_of_pair[c["pair"]], c["grad"], c["gves"], c["gvid"], nverts)
    return rows, -c["V_pair"][hit], nverts


def _dense_M(m, t, nverts):
    """The block-diagonal M written out: per vesicle m_i I + t_i (1 1^T (x) I_3)
    over its 3 n_v coordinates (point-major, x y z)."""
    blocks = []
    for v, nv in enumerate(nverts):
        blk = m[v] * np.eye(3 * nv)
        if t is not None:
            blk += t[v] * np.kron(np.ones((nv, nv)), np.eye(3))
        blocks.append(blk)
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    o = 0
    for b in blocks:
        M[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return M


@pytest.mark.parametrize("with_t", [False, True])
def test_alg3_equals_j_m_jt(orc, with_t):
    """Alg. 3's per-vesicle accumulation equals the matrix product J M J^T
    with M written out densely."""
    sc = G.scene_small((4, 4, 2), p=3, seed=6, periodic=True)
    rows, q, nverts = _scene_lcp(orc, sc)
    assert len(rows) >= 30
    m = np.linspace(0.5, 2.0, sc.n)
    t = np.linspace(0.05, 0.01, sc.n) if with_t else None
    B = L.lcp_matrix_alg3(rows, m, t)
    J, offs = L.dense_jacobian(rows, nverts)
    ref = J @ _dense_M(m, t, nverts) @ J.T
    assert np.allclose(B, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert np.allclose(B, B.T, rtol=1e-12)
    # every pair of volumes sharing a vesicle couples through the translation term
    share = np.array([[bool(set(a) & set(b)) for b in rows] for a in rows])
    if with_t:
        assert np.array_equal(B != 0, share)
    assert np.all(np.linalg.eigvalsh(B) > -1e-12 * np.abs(B).max())


def test_scene_lcp_kkt(orc):
    """The contact LCP of a small periodic suspension: lambda >= 0,
    -V + B lambda >= 0 (the interference removed to first order),
    complementarity."""
    sc = G.scene_small((4, 4, 2), p=3, seed=6, periodic=True)
    rows, q, _ = _scene_lcp(orc, sc)
    assert len(rows) >= 30
    B = L.lcp_matrix_alg3(rows, np.ones(sc.n))
    x, it, res = L.minmap_newton(B, q)
    w = B @ x + q
    scale = np.abs(q).max()
    assert res <= 1e-12 * max(scale, 1.0)
    assert np.all(x >= 0) and np.all(w >= -1e-12 * scale)
    assert abs(float(x @ w)) <= 1e-10 * scale * max(np.abs(x).max(), 1.0)
    assert (x > 0).sum() >= len(q) // 2      # most interfering pairs need a contact force
