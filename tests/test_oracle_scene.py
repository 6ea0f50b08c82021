"""Scene-level pins of the oracle (Alg. 2 over all vesicle pairs): closed
forms, brute force and invariants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1812_04719_gb300 import scenegen as G
from tests.oracle_scene import contact_keys, run_scene, synth_scene


def two_spheres(p, gap, closing, direction, R=1.0):
    d = np.asarray(direction, float); d /= np.linalg.norm(d)
    c1, c2 = np.zeros(3), d * (2 * R + gap)
    k1 = G.ellipsoid_coef(p, c1, R * np.eye(3))
    k2 = G.ellipsoid_coef(p, c2, R * np.eye(3))
    k2e = G.rigid_motion(k2, np.eye(3), -closing * d, c2)
    return G._pack("two spheres", [p, p], [np.stack([k1, k1]), np.stack([k2, k2e])], np.zeros(3),
                   np.stack([c1, c2]))


@pytest.mark.parametrize("p", [4, 8, 16])
def test_two_spheres_head_on(orc, p):
    """Analytic contact time of the spheres tau_s = gap / closing; the inscribed
    mesh touches later, by at most its sagitta over the closing distance."""
    gap, closing = 0.05, 0.1
    sc = two_spheres(p, gap, closing, [0.3, 0.5, 0.81])
    _, c = run_scene(sc)
    assert len(c["pair"]) > 0
    tau_s = gap / closing
    sag = 2 * (1 - math.cos(math.pi / (2 * p))) * 2  # both surfaces, diagonal-length chords
    tmin = c["tau"].min()
    assert tau_s <= tmin <= tau_s + sag / closing
    assert np.all(c["V"] >= 0)


def test_two_spheres_converge(orc):
    gap, closing = 0.05, 0.1
    errs = []
    for p in (4, 8, 16):
        sc = two_spheres(p, gap, closing, [0.3, 0.5, 0.81])
        _, c = run_scene(sc, include_ee=False)
        errs.append(c["tau"].min() - gap / closing)
    assert errs[0] > errs[1] > errs[2] >= 0


def test_separating_vesicles_have_no_contacts(orc):
    sc = two_spheres(4, 0.05, -0.3, [1, 0.2, 0.1])
    _, c = run_scene(sc)
    assert len(c["pair"]) == 0 and np.all(c["V_pair"] == 0)


def test_bruteforce_equals_pruned(orc):
    """No-pruning mode gives the identical contact list (keys and tau bits)."""
    sc = G.scene_small((2, 1, 1), p=3, seed=3)
    Xs, c1 = run_scene(sc, prune=True)
    _, c2 = run_scene(sc, Xs=Xs, prune=False)
    assert len(c1["pair"]) > 0
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(c1[k], c2[k])
    assert np.array_equal(c1["tau"].view(np.int64), c2["tau"].view(np.int64))
    assert c2["counts"][1] > c1["counts"][1]


def test_permutation_invariance(orc):
    sc = G.scene_small((4, 4, 2), p=2, seed=5, periodic=True)
    Xs, c = run_scene(sc)
    perm = np.random.default_rng(0).permutation(sc.n)
    inv = np.argsort(perm)
    Xp = [Xs[perm[k]] for k in range(sc.n)]
    scp = G._pack("perm", sc.p[perm], [sc.coef_of(v).copy() for v in perm], sc.L, sc.centers[perm])
    _, cp = run_scene(scp, Xs=Xp)

    def canon(c, relabel):
        out = {}
        for r, (i, j, sx, sy, sz) in enumerate(c["pairs"]):
            a, b = relabel[i], relabel[j]
            s = (sx, sy, sz)
            if a > b:
                a, b, s = b, a, (-sx, -sy, -sz)
            out[(a, b) + s] = c["V_pair"][r]
        return out
    A = canon(c, np.arange(sc.n))
    B = canon(cp, perm)
    assert set(A) == set(B)
    for k in A:
        assert abs(A[k] - B[k]) <= 1e-12 * max(abs(A[k]), 1e-300)
    assert sum(v > 0 for v in A.values()) > 0


def test_rigid_motion_of_scene(orc):
    """Integer translation and a rotation of the whole (free-space) scene leave
    every pair's V unchanged to 1e-10 relative."""
    sc = G.two_vesicles(p=4, seed=9)
    Xs, c = run_scene(sc)
    rng = np.random.default_rng(1)
    R = G.random_rotation(rng)
    t = np.array([3.0, -2.0, 5.0])
    Xr = [np.einsum("ij,tjn->tin", R, X) + t[None, :, None] for X in Xs]
    _, cr = run_scene(sc, Xs=Xr)
    assert c["V_pair"][0] > 0
    assert abs(cr["V_pair"][0] - c["V_pair"][0]) < 1e-10 * c["V_pair"][0]


def test_volume_zero_iff_no_contact(orc):
    sc = G.scene_small((4, 4, 2), p=2, seed=5, periodic=True)
    _, c = run_scene(sc)
    has = np.zeros(len(c["pairs"]), bool)
    has[c["pair"]] = True
    assert np.all((c["V_pair"] > 0) == has)


def test_gradient_wrt_sh_coefficients(orc):
    """d(sum V)/d(coef of X1) = S^T (dV/dX1) against central differences in the
    coefficients (h = 1e-6) where the contact list does not change."""
    sc = G.two_vesicles(p=3, seed=2, approach=0.15)
    Xs, c = run_scene(sc)
    assert len(c["pair"]) > 0
    p, P = 3, 6
    nv = G.nverts(P)
    gX = np.zeros((2, 3, nv))
    for k in range(len(c["pair"])):
        for q in range(4):
            gX[c["gves"][k, q], :, c["gvid"][k, q]] += c["grad"][k, q]
    gcoef = np.stack([[O.synth_adjoint(p, P, gX[v, d]) for d in range(3)] for v in range(2)])
    rng = np.random.default_rng(0)
    h = 1e-6
    checked = 0
    keys0 = contact_keys(c)
    for _ in range(30):
        v, d, q = rng.integers(2), rng.integers(3), rng.integers((p + 1) ** 2)
        vals = []
        for s in (+1, -1):
            coef = sc.coef.copy()
            coef[sc.coef_off[v] + (1 * 3 + d) * (p + 1) ** 2 + q] += s * h
            sc2 = G._pack("fd", sc.p, [coef[sc.coef_off[u]:sc.coef_off[u] + 6 * (p + 1) ** 2].reshape(2, 3, -1)
                                       for u in range(2)], sc.L, sc.centers)
            _, c2 = run_scene(sc2)
            if contact_keys(c2) != keys0:
                break
            vals.append(c2["V_pair"].sum())
        if len(vals) < 2:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gcoef[v, d, q]) < 1e-6 * max(1.0, np.abs(gcoef).max())
        checked += 1
    assert checked >= 10
