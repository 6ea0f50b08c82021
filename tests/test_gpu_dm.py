"""Contact detection with minimum separation d_m > 0 on the GPU (Eq. 3.1, the
degree-six equation; boxes widened by d_m; the certified FP32 rejection, proved
for the cubic only, bypassed) against the oracle on the oracle's vertices:
candidate pairs, the primitive pairs tested, every contact (keys, contact
times and weights bit for bit), V within 1e-10 and dV/dX1 within 1e-9."""
import dataclasses

import numpy as np
import pytest

from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import gpu_pairs_rows, run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices
from tests.test_gpu_parity import SCENES

pytestmark = pytest.mark.gpu


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


@pytest.mark.parametrize("d_m", [0.005, 0.03])
@pytest.mark.parametrize("name", ["cluster_p4", "periodic_p3", "uneven_p234"])
@pytest.mark.parametrize("precision", [S.STIV_FP64, S.STIV_MIXED])
def test_dm_matches_oracle(orc, name, d_m, precision):
    sc = dataclasses.replace(SCENES[name](), d_m=d_m)
    X = oracle_vertices(sc)
    g = run_gpu_on(sc, X, precision=precision, pair_cap=512, contact_cap=1 << 15)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(x, sc.d_m) for x in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, d_m=d_m)
    assert len(c["pair"]) > 20
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.array_equal(bits(g["w"]), bits(c["w"]))
    assert g["counts"][S.C_PRIM] == c["counts"][1]
    assert g["counts"][S.C_DEGEN] == c["counts"][2]
    assert np.all(np.abs(g["V"] - c["V"]) <= 1e-10 * np.abs(c["V"]))
    scale = np.abs(c["grad"]).reshape(len(c["pair"]), -1).max(axis=1)
    err = np.abs(g["grad"] - c["grad"]).reshape(len(c["pair"]), -1).max(axis=1)
    assert np.all(err <= 1e-9 * scale + 1e-300), float((err / scale).max())


def test_dm_graph_replay_and_more_contacts():
    """The whole step (graph replay) with d_m > 0 gives the eager results, and
    finds more contacts than d_m = 0 on the same vertices."""
    sc0 = SCENES["periodic_p3"]()
    sc = dataclasses.replace(sc0, d_m=0.03)
    X = oracle_vertices(sc0)
    e = run_gpu_on(sc, X)
    r = run_gpu_on(sc, X, use_graph=True, replays=3)
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(e[k], r[k]), k
    assert np.array_equal(bits(e["tau"]), bits(r["tau"]))
    z = run_gpu_on(sc0, X)
    assert len(e["pair"]) > len(z["pair"])


@pytest.mark.parametrize("precision", [S.STIV_FP64, S.STIV_MIXED])
def test_dm_band_filter_is_exact(precision):
    """The certified FP32 band rejection changes no result: with and without
    it (exact_only) the contact lists, times, weights and counts agree bit for
    bit on the 144-vesicle piece of the 58% lattice, and it keeps most pairs
    away from the FP64 degree-six test (those certainly out of the band over
    the step, and those outside the primitive wherever they may be in it)."""
    from paper_1812_04719_gb300 import scenegen as G
    dm = 1.1 * (0.009 / 1.136) * G.R0_PAPER
    sc = dataclasses.replace(G.scene_lattice58((6, 6, 2)), d_m=dm)
    X = oracle_vertices(sc)
    kw = dict(precision=precision, pair_cap=2048, contact_cap=1 << 18)
    f = run_gpu_on(sc, X, **kw)
    x = run_gpu_on(sc, X, eng=S.Stiv.for_scene(sc, precision=precision, pair_cap=2048, contact_cap=1 << 18,
                                                exact_only=True), **kw)
    assert f["counts"][S.C_VF] + f["counts"][S.C_EE] > 10000
    for k in ("i", "j", "shift", "pair", "type", "a", "b"):
        assert np.array_equal(f[k], x[k]), k
    assert np.array_equal(bits(f["tau"]), bits(x["tau"]))
    assert np.array_equal(bits(f["w"]), bits(x["w"]))
    for c in (S.C_PAIRS, S.C_PRIM, S.C_VF, S.C_EE, S.C_CPAIRS, S.C_DEGEN):
        assert f["counts"][c] == x["counts"][c], c
    assert f["counts"][S.C_EXACT] < 0.2 * x["counts"][S.C_EXACT]
    # the operation count: every pair that reaches the degree-six test costs at
    # least its set-up (displacements 12, coefficients and derivatives 172)
    for r in (f, x):
        assert r["counts"][S.C_FLOPS] >= 184 * r["counts"][S.C_EXACT] > 0
    print(f"band filter: {f['counts'][S.C_EXACT]} of {x['counts'][S.C_EXACT]} pairs reach the FP64 test")
