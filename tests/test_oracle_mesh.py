"""Pins of the oracle's triangulation of the (P+1) x 2P grid (Sec. 3.1.2, Fig. 3)."""
import collections

import numpy as np
import pytest

from paper_1812_04719_gb300 import scenegen as G


@pytest.mark.parametrize("P", [2, 4, 16, 24, 32])
def test_counts_and_closed_manifold(orc, P):
    tri = orc.triangles(P)
    edg = orc.edges(P)
    nv, nf, ne = 2 * P * (P + 1) + 2, 4 * P * P + 4 * P, 6 * P * P + 6 * P
    assert tri.shape == (nf, 3) and edg.shape == (ne, 2)
    assert tri.min() == 0 and tri.max() == nv - 1
    assert nv - ne + nf == 2  # genus 0
    # every directed edge once (consistent orientation), every undirected edge twice
    directed = collections.Counter()
    for t in tri:
        for k in range(3):
            directed[(int(t[k]), int(t[(k + 1) % 3]))] += 1
    assert max(directed.values()) == 1
    und = collections.Counter(tuple(sorted(e)) for e in directed)
    assert all(v == 2 for v in und.values())
    assert sorted(und) == [tuple(e) for e in edg.tolist()]
    assert np.all(edg[:, 0] < edg[:, 1])


@pytest.mark.parametrize("p", [4, 16])
def test_outward_orientation_and_volume(orc, p):
    """On a synthesized prolate vesicle every triangle normal points away from
    the centre and the enclosed volume converges to the ellipsoid volume."""
    P = 2 * p
    a, b = G.prolate_axes()
    coef = G.ellipsoid_coef(p, np.zeros(3), np.diag([b, b, a]))
    X = np.stack([orc.synth(p, P, coef[k]) for k in range(3)]).T
    tri = orc.triangles(P)
    x0, x1, x2 = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    n = np.cross(x1 - x0, x2 - x0)
    cen = (x0 + x1 + x2) / 3
    assert np.all(np.einsum("ij,ij->i", n, cen) > 0)
    vol = np.einsum("ij,ij->i", x0, np.cross(x1, x2)).sum() / 6
    exact = 4 / 3 * np.pi * a * b * b
    assert 0 < exact - vol < (0.08 if P < 16 else 0.006) * exact  # inscribed mesh, converging
