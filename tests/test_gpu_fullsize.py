"""Parity at the benchmark's full sizes: the 1440-vesicle 58% lattice workload
(p = 16 -> 32) and the 4096-vesicle 40% workload of uneven orders (p in
{8, 12, 16}), run as the benchmark runs them (graph replay of the whole
step).  The upsampled vertices are compared with the oracle's synthesis; the
detection is then replayed on the oracle's vertices, and its whole
candidate-pair list is compared with the oracle's all-pairs box test bit for
bit; contacts, volumes and gradient rows are compared on a sample of vesicle
pairs that the oracle recomputes one by one.  The 4096 workload's whole
contact lists are compared in both forms (test_whole_lists_4096, about a
minute and a half of the oracle on 16 host cores per form); the 1440
workload's are in test_gpu_fulllist.py."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import assert_whole_list, gpu_pairs_rows, oracle_scene, run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices

pytestmark = pytest.mark.gpu


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


@pytest.fixture(scope="module", params=[("1440", S.STIV_FP64), ("1440", S.STIV_MIXED), ("4096", S.STIV_MIXED)],
                ids=["1440-fp64", "1440-mixed", "4096-mixed"])
def full(request):
    name, prec = request.param
    sc = G.scene_1440() if name == "1440" else G.scene_4096()
    Xo = oracle_vertices(sc)
    eng = S.Stiv.for_scene(sc, precision=prec, pair_cap=8192, contact_cap=1 << 20)
    ds = S.DeviceScene.from_scene(sc, precision=prec)
    for _ in range(3):   # capture, then replays
        eng.step(ds, grad=True, use_graph=True)
    torch.cuda.synchronize()
    up = ds.verts.double().cpu().numpy()
    g = run_gpu_on(sc, Xo, precision=prec, grad=True, use_graph=True, replays=3, eng=eng)
    return sc, g, up, Xo, prec


def mixed_vertex_bound(sc, Xo):
    """The MIXED synthesis bound per vertex coordinate of field (vesicle, time,
    coordinate) with coefficients a_q: 2^-23 |X| + 2^-19 sum_{q>0} |a_q| Ymax,
    Ymax = sqrt((2p+1) / (2 pi)) (3xTF32 split products, FP32 accumulation)."""
    out = np.empty_like(Xo)
    for v, (o, n) in enumerate(zip(sc.vert_off(), sc.vert_sizes())):
        p = int(sc.p[v])
        a1 = np.abs(sc.coef_of(v)[:, :, 1:]).sum(axis=-1)[:, :, None]
        X = Xo[o:o + n].reshape(2, 3, -1)
        out[o:o + n] = (2.0 ** -23 * np.abs(X) + 2.0 ** -19 * a1 * np.sqrt((2 * p + 1) / (2 * np.pi))).ravel()
    return out


def test_upsample_full(full):
    """Synthesis at p -> 2p of every vesicle: FP64 within 1e-13 of the
    oracle's (relative to the largest coordinate), MIXED (tensor cores, FP32
    output) within its per-vertex bound."""
    sc, g, up, Xo, prec = full
    if prec == S.STIV_FP64:
        assert np.abs(up - Xo).max() <= 1e-13 * np.abs(Xo).max()
    else:
        assert np.all(np.abs(up - Xo) <= mixed_vertex_bound(sc, Xo))


def test_candidate_pairs_full(orc, full):
    sc, g = full[:2]
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert len(pairs) > 5000
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    assert g["counts"][S.C_STATUS] == 0


def test_sampled_pairs_contacts_volumes_gradients(orc, full):
    sc, g = full[:2]
    Xs = verts_list(sc, g["verts"])
    rows = gpu_pairs_rows(g)
    rng = np.random.default_rng(11)
    hit = np.nonzero(g["V_pair"] > 0)[0]
    miss = np.nonzero(g["V_pair"] == 0)[0]
    sample = np.sort(np.concatenate([rng.choice(hit, 24, replace=False), rng.choice(miss, 8, replace=False)]))
    c = orc.contacts(sc.P, Xs, rows[sample], sc.L, sc.eps * sc.dt, grad=True)
    n_checked = 0
    for k, r in enumerate(sample):
        gm = g["pair"] == r
        cm = c["pair"] == k
        for key in ("type", "a", "b"):
            assert np.array_equal(g[key][gm], c[key][cm]), (r, key)
        assert np.array_equal(bits(g["tau"][gm]), bits(c["tau"][cm]))
        assert np.array_equal(bits(g["w"][gm]), bits(c["w"][cm]))
        assert abs(g["V_pair"][r] - c["V_pair"][k]) <= 1e-10 * abs(c["V_pair"][k])
        assert np.all(np.abs(g["V"][gm] - c["V"][cm]) <= 1e-10 * np.abs(c["V"][cm]))
        gr, cr = g["grad"][gm], c["grad"][cm]
        if len(cr):
            scale = np.abs(cr).reshape(len(cr), -1).max(axis=1)
            err = np.abs(gr - cr).reshape(len(cr), -1).max(axis=1)
            assert np.all(err <= 1e-9 * scale + 1e-300)
            assert np.array_equal(g["gvid"][gm], c["gvid"][cm])
            assert np.array_equal(g["gves"][gm], c["gves"][cm])
        n_checked += int(gm.sum())
    assert n_checked > 1000


@pytest.mark.parametrize("name,prec", [("64", S.STIV_FP64), ("64", S.STIV_MIXED), ("256", S.STIV_FP64),
                                       ("256", S.STIV_MIXED)])
def test_whole_scene_lists(orc, name, prec):
    """The 64-vesicle 30% workload (random orientations, p = 16 -> 32) and the
    256-vesicle 50% workload (p = 12 -> 24): every candidate pair and every
    contact (keys, contact times and weights bit for bit), V per pair within
    1e-10, against the oracle run on the same vertices (its own synthesis, in
    the form's vertex type)."""
    sc = G.scene_64() if name == "64" else G.scene_256()
    g = run_gpu_on(sc, oracle_vertices(sc), precision=prec, grad=False, use_graph=True, replays=2, pair_cap=4096,
                   contact_cap=1 << 18)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=False)
    assert len(c["pair"]) > 0
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.array_equal(bits(g["w"]), bits(c["w"]))
    assert np.all(np.abs(g["V_pair"] - c["V_pair"]) <= 1e-10 * np.abs(c["V_pair"]))
    assert g["counts"][S.C_PRIM] == c["counts"][1]


def test_dm_sampled_pairs_1440(orc):
    """The 1440-vesicle workload with minimum separation d_m (the paper's
    0.009 at R0 = 1.136 scaled to R0 and inflated by 1 + 2 alpha, the degree-six
    test), MIXED form, graph replay on the oracle's vertices: the candidate
    list bit for bit, and contacts, volumes and gradient rows on a sample of
    pairs the oracle recomputes."""
    import dataclasses
    dm = 1.1 * (0.009 / 1.136) * G.R0_PAPER
    sc = dataclasses.replace(G.scene_1440(), d_m=dm)
    g = run_gpu_on(sc, oracle_vertices(sc), precision=S.STIV_MIXED, grad=True, use_graph=True, replays=3,
                   pair_cap=8192, contact_cap=1 << 20)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    rng = np.random.default_rng(12)
    hit = np.nonzero(g["V_pair"] > 0)[0]
    miss = np.nonzero(g["V_pair"] == 0)[0]
    sample = np.sort(np.concatenate([rng.choice(hit, 16, replace=False), rng.choice(miss, 8, replace=False)]))
    c = orc.contacts(sc.P, Xs, pairs[sample], sc.L, sc.eps * sc.dt, grad=True, d_m=dm)
    n_checked = 0
    for k, r in enumerate(sample):
        gm = g["pair"] == r
        cm = c["pair"] == k
        for key in ("type", "a", "b"):
            assert np.array_equal(g[key][gm], c[key][cm]), (r, key)
        assert np.array_equal(bits(g["tau"][gm]), bits(c["tau"][cm]))
        assert np.array_equal(bits(g["w"][gm]), bits(c["w"][cm]))
        assert abs(g["V_pair"][r] - c["V_pair"][k]) <= 1e-10 * abs(c["V_pair"][k])
        gr, cr = g["grad"][gm], c["grad"][cm]
        if len(cr):
            scale = np.abs(cr).reshape(len(cr), -1).max(axis=1)
            err = np.abs(gr - cr).reshape(len(cr), -1).max(axis=1)
            assert np.all(err <= 1e-9 * scale + 1e-300)
        n_checked += int(gm.sum())
    assert n_checked > 500


@pytest.fixture(scope="module")
def scene4096():
    sc = G.scene_4096()
    return sc, oracle_vertices(sc)


@pytest.fixture(scope="module")
def oracle4096(orc, scene4096):
    sc, Xo = scene4096
    return oracle_scene(orc, sc, Xo)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [S.STIV_FP64, S.STIV_MIXED], ids=["fp64", "mixed"])
def test_whole_lists_4096(orc, scene4096, oracle4096, prec):
    """The batched workload of uneven orders (4096 vesicles at 40%, p in {8,
    12, 16}, 545M exact-box primitive pairs, 1.33M contacts), graph replay on
    the oracle's vertices (FP64, or rounded to FP32 for the MIXED form):
    every candidate pair, every contact (keys, contact time and weights bit
    for bit), V per contact and per pair within 1e-10, every gradient row
    within 1e-9, the exact-box pair count, against the oracle's Alg. 2 over
    the whole scene on the same values."""
    sc, Xo = scene4096
    g = run_gpu_on(sc, Xo, precision=prec, grad=True, use_graph=True, replays=3, pair_cap=1 << 15,
                   contact_cap=1 << 21)
    c = oracle4096 if prec == S.STIV_FP64 else oracle_scene(orc, sc, g["verts"])
    assert_whole_list(g, c)
