"""CUDA path vs the FP64 oracle, through the C-ABI (pytest -m gpu)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.golden_table3 import load as load_table3
from tests.gpu_run import gpu_pairs_rows, run_gpu, run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices

pytestmark = pytest.mark.gpu


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


@pytest.mark.parametrize("P", [2, 4, 6, 16, 24, 32, 64])
def test_mesh_topology(orc, P):
    nf, ne = 4 * P * P + 4 * P, 6 * P * P + 6 * P
    tri = torch.zeros(nf, 3, dtype=torch.int32, device="cuda")
    edg = torch.zeros(ne, 2, dtype=torch.int32, device="cuda")
    S.stiv_mesh_topology(P, tri.data_ptr(), edg.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(tri.cpu().numpy(), orc.triangles(P))
    assert np.array_equal(edg.cpu().numpy(), orc.edges(P))


def test_sort_table3_fixture():
    """Alg. 1's check-point sort on the GPU: Table 3's keys and payloads."""
    t = load_table3()
    n = 8
    keys = torch.tensor(t["unsorted_M"], dtype=torch.int64, device="cuda")
    vals = torch.tensor(t["unsorted_Ic"], dtype=torch.int32, device="cuda")
    ko = torch.zeros_like(keys); vo = torch.zeros_like(vals)
    nb = S.stiv_sort_scratch_bytes(n)
    scr = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    S.stiv_sort_pairs(torch.cuda.current_stream().cuda_stream, n, 3, keys.data_ptr(), vals.data_ptr(),
                      ko.data_ptr(), vo.data_ptr(), scr.data_ptr(), nb)
    torch.cuda.synchronize()
    assert ko.cpu().tolist() == t["sorted_M"]
    assert vo.cpu().tolist() == t["sorted_Ic"]
    icb = np.array(t["unsorted_Icb"])[np.array(vo.cpu().tolist()) - 1]
    assert icb.tolist() == t["scatter_Icb"]


@pytest.mark.parametrize("n,bits_", [(1, 8), (1000, 12), (70000, 40), (300000, 64), (3000001, 35)])
def test_sort_random_stable(n, bits_):
    rng = np.random.default_rng(n)
    k = rng.integers(0, 2 ** min(bits_, 62), size=n, dtype=np.int64)
    k[: n // 3] = k[n // 3: 2 * (n // 3)]  # many ties
    keys = torch.tensor(k, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko = torch.zeros_like(keys); vo = torch.zeros_like(vals)
    nb = S.stiv_sort_scratch_bytes(n)
    scr = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    S.stiv_sort_pairs(torch.cuda.current_stream().cuda_stream, n, bits_, keys.data_ptr(), vals.data_ptr(),
                      ko.data_ptr(), vo.data_ptr(), scr.data_ptr(), nb)
    torch.cuda.synchronize()
    order = np.argsort(k, kind="stable")
    assert np.array_equal(ko.cpu().numpy(), k[order])
    assert np.array_equal(vo.cpu().numpy(), order.astype(np.int32))
    assert np.array_equal(keys.cpu().numpy(), k)  # input left intact


SCENES = {
    "pair_p8": lambda: G.scene_pair(),
    "cluster_p4": lambda: G.scene_small((2, 2, 1), p=4, seed=3),
    "periodic_p2": lambda: G.scene_small((4, 4, 2), p=2, seed=5, periodic=True),
    "periodic_p3": lambda: G.scene_small((4, 4, 2), p=3, seed=6, periodic=True),
}


def uneven_scene():
    sc = G.scene_small((4, 4, 2), p=2, seed=8, periodic=True)
    rng = np.random.default_rng(1)
    ps = rng.choice([2, 3, 4], size=sc.n)
    coefs = []
    for v in range(sc.n):
        c = sc.coef_of(v)
        p = int(ps[v])
        out = np.zeros((2, 3, (p + 1) ** 2))
        k = min(c.shape[-1], out.shape[-1])
        out[:, :, :k] = c[:, :, :k]
        coefs.append(out)
    return G._pack("uneven", ps, coefs, sc.L, sc.centers)


SCENES["uneven_p234"] = uneven_scene


@pytest.mark.parametrize("name", list(SCENES))
def test_upsample_matches_oracle(orc, name):
    sc = SCENES[name]()
    g = run_gpu(sc, grad=False)
    Xo = np.concatenate([orc.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)).ravel() for v in range(sc.n)])
    scale = np.abs(Xo).max()
    assert np.abs(g["verts"] - Xo).max() < 1e-13 * max(scale, 1.0)


@pytest.mark.parametrize("name", list(SCENES) + ["lattice_144_p16"])
def test_upsample_mixed_tensor_cores(orc, name):
    """STIV_MIXED synthesis (tensor cores, 3xTF32 products, FP32 accumulation,
    degree-0 term added in the epilogue) against the FP64 oracle.  Bound per
    vertex of field (vesicle, time, coordinate) with coefficients a_q:
    2^-23 |X| (FP32 result and degree-0 rounding) + 2^-19 sum_{q>0} |a_q| Ymax,
    Ymax = sqrt((2p+1) / (2 pi)) >= |Y_q| (each split product keeps a relative
    error near 2^-22; FP32 accumulation over the terms)."""
    sc = G.scene_lattice58((6, 6, 2)) if name == "lattice_144_p16" else SCENES[name]()
    g = run_gpu(sc, precision=S.STIV_MIXED, grad=False, pair_cap=2048, contact_cap=1 << 17)
    worst = 0.0
    offs = sc.vert_off()
    for v in range(sc.n):
        p, P = int(sc.p[v]), int(sc.P[v])
        Xo = orc.synth_vesicle(p, P, sc.coef_of(v))
        Xg = g["verts"][offs[v]:offs[v] + Xo.size].reshape(Xo.shape)
        a1 = np.abs(sc.coef_of(v)[:, :, 1:]).sum(axis=-1)[:, :, None]
        bound = 2.0 ** -23 * np.abs(Xo) + 2.0 ** -19 * a1 * np.sqrt((2 * p + 1) / (2 * np.pi))
        assert np.all(np.abs(Xg - Xo) <= bound), v
        worst = max(worst, float((np.abs(Xg - Xo) / bound).max()))
    print(f"mixed synthesis: max error / bound = {worst:.3f}")


@pytest.mark.parametrize("name", list(SCENES))
def test_detect_bit_exact(orc, name):
    """Candidate pairs and contacts (keys, tau and weights bit for bit) equal
    the oracle's on the same vertices (the oracle's synthesis); the counted
    primitive pairs too."""
    sc = SCENES[name]()
    g = run_gpu_on(sc, oracle_vertices(sc))
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt)
    assert len(c["pair"]) > 0
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.array_equal(bits(g["w"]), bits(c["w"]))
    assert g["counts"][S.C_PRIM] == c["counts"][1]
    assert g["counts"][S.C_DEGEN] == c["counts"][2]
    assert g["counts"][S.C_CPAIRS] == int((c["V_pair"] > 0).sum())


@pytest.mark.parametrize("name", ["cluster_p4", "periodic_p3", "uneven_p234"])
def test_operation_count_exact_mode(orc, name):
    """With the FP32 rejection off every primitive pair of the exact box test
    reaches the FP64 contact test, so the operations the kernel counts equal
    the oracle's count of the same procedure (the roofline's algorithmic
    work), operation for operation."""
    sc = SCENES[name]()
    eng = S.Stiv.for_scene(sc, pair_cap=256, contact_cap=4096, exact_only=True)
    g = run_gpu_on(sc, oracle_vertices(sc), eng=eng)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt)
    assert g["counts"][S.C_PRIM] == c["counts"][1]
    assert g["counts"][S.C_EXACT] == c["counts"][1]
    assert g["counts"][S.C_FLOPS] == c["counts"][3]


@pytest.mark.parametrize("name", list(SCENES))
def test_stiv_and_gradient(orc, name):
    sc = SCENES[name]()
    g = run_gpu_on(sc, oracle_vertices(sc))
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True)
    assert np.array_equal(g["pair"], c["pair"])
    assert np.all(np.abs(g["V"] - c["V"]) <= 1e-10 * np.abs(c["V"]) + 1e-300)
    assert np.all(np.abs(g["V_pair"] - c["V_pair"]) <= 1e-10 * np.abs(c["V_pair"]) + 1e-300)
    assert np.array_equal(g["gves"], c["gves"]) and np.array_equal(g["gvid"], c["gvid"])
    gn = np.abs(c["grad"]).reshape(len(c["pair"]), -1).max(axis=1)
    err = np.abs(g["grad"] - c["grad"]).reshape(len(c["pair"]), -1).max(axis=1)
    assert np.all(err <= 1e-9 * gn + 1e-300), (err / gn).max()


def test_graph_replay_matches_eager():
    sc = SCENES["periodic_p3"]()
    g1 = run_gpu(sc)
    eng = g1["eng"]
    ds = g1["ds"]
    for _ in range(3):
        r = eng.step(ds, grad=True, use_graph=True)
    torch.cuda.synchronize()
    assert np.array_equal(r["tau"].cpu().numpy().view(np.int64), g1["tau"].view(np.int64))
    assert np.array_equal(r["a"].cpu().numpy(), g1["a"])
    assert np.array_equal(r["V_pair"].cpu().numpy(), g1["V_pair"])


@pytest.mark.parametrize("name", ["cluster_p4", "uneven_p234"])
def test_adjoint_matches_oracle(orc, name):
    sc = SCENES[name]()
    g = run_gpu(sc)
    ds = g["ds"]
    rng = np.random.default_rng(3)
    gX = torch.tensor(rng.normal(size=ds.verts.numel()), dtype=torch.float64, device="cuda")
    gc = torch.zeros_like(ds.coef)
    S.stiv_grad_to_coef(g["eng"].h, torch.cuda.current_stream().cuda_stream, ds.n, ds.p_max, ds.p.data_ptr(),
                        ds.coef_off.data_ptr(), ds.vert_off.data_ptr(), gX.data_ptr(), gc.data_ptr())
    torch.cuda.synchronize()
    gXh = gX.cpu().numpy()
    gch = gc.cpu().numpy()
    vo = sc.vert_off()
    for v in range(sc.n):
        p, P = int(sc.p[v]), int(sc.P[v])
        nv = G.nverts(P)
        blk = gXh[vo[v]:vo[v] + 6 * nv].reshape(2, 3, nv)
        got = gch[sc.coef_off[v]:sc.coef_off[v] + 6 * (p + 1) ** 2].reshape(2, 3, -1)
        assert np.all(got[0] == 0)
        for d in range(3):
            ref = orc.synth_adjoint(p, P, blk[1, d])
            assert np.abs(got[1, d] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("name", ["cluster_p4", "uneven_p234", "lattice_144_p16"])
def test_adjoint_mixed_tensor_cores(orc, name):
    """STIV_MIXED adjoint (tensor cores, 3xTF32 products, FP32 accumulation over
    the vertices) against the FP64 oracle adjoint.  Bound per coefficient:
    2^-12 sum_rows |Y| |gX| <= 2^-12 Ymax sum_rows |gX| (accumulation of n_v
    terms in FP32 at worst n_v 2^-24 of their absolute sum, plus the split
    products' 2^-22 each); the measured ratio is printed."""
    sc = G.scene_lattice58((6, 6, 2)) if name == "lattice_144_p16" else SCENES[name]()
    g = run_gpu(sc, precision=S.STIV_MIXED, pair_cap=2048, contact_cap=1 << 17)
    eng = g["eng"]
    ds = g["ds"]
    rng = np.random.default_rng(4)
    gX = torch.tensor(rng.normal(size=ds.verts.numel()), dtype=torch.float64, device="cuda")
    gc = torch.full_like(ds.coef, 7.0)
    S.stiv_grad_to_coef(eng.h, torch.cuda.current_stream().cuda_stream, ds.n, ds.p_max, ds.p.data_ptr(),
                        ds.coef_off.data_ptr(), ds.vert_off.data_ptr(), gX.data_ptr(), gc.data_ptr())
    torch.cuda.synchronize()
    gXh, gch = gX.cpu().numpy(), gc.cpu().numpy()
    vo = sc.vert_off()
    worst = 0.0
    for v in range(sc.n):
        p, P = int(sc.p[v]), int(sc.P[v])
        nv = G.nverts(P)
        blk = gXh[vo[v]:vo[v] + 6 * nv].reshape(2, 3, nv)
        got = gch[sc.coef_off[v]:sc.coef_off[v] + 6 * (p + 1) ** 2].reshape(2, 3, -1)
        assert np.all(got[0] == 0)
        ymax = np.sqrt((2 * p + 1) / (2 * np.pi))
        for d in range(3):
            ref = orc.synth_adjoint(p, P, blk[1, d])
            scale = ymax * np.abs(blk[1, d]).sum()
            err = np.abs(got[1, d] - ref).max()
            assert err <= 2.0 ** -12 * scale, (v, d, err, scale)
            worst = max(worst, err / scale)
    print(f"mixed adjoint: max error / (Ymax sum|gX|) = {worst:.3g}")


def test_mixed_precision_lists(orc):
    """MIXED: FP32 vertices (the tensor-core synthesis within 4e-7 of the
    oracle's); the FP64 contact arithmetic on FP32 vertices is bit-identical
    to the oracle run on the same (widened) vertices, here the oracle's
    synthesis rounded to FP32."""
    sc = SCENES["periodic_p3"]()
    g_up = run_gpu(sc, precision=S.STIV_MIXED)
    Xo = oracle_vertices(sc)
    assert np.abs(g_up["verts"] - Xo).max() < 4e-7 * np.abs(Xo).max()
    g = run_gpu_on(sc, Xo, precision=S.STIV_MIXED)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt)
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.all(np.abs(g["V"] - c["V"]) <= 1e-10 * np.abs(c["V"]))


def test_contact_order_large_segments():
    """Pairs with more contacts than one shared-memory sort chunk are merged
    correctly: the contact list is sorted by (pair, type, a, b) and unique."""
    sc = G.two_vesicles(p=16, seed=4, gap=0.02, approach=1.5)
    g = run_gpu(sc, grad=False, contact_cap=1 << 16)
    n = len(g["pair"])
    assert n > 4096  # more than one shared-memory chunk (4096 entries)
    key = (g["pair"].astype(np.int64) << 32) | (g["type"].astype(np.int64) << 30) | (g["a"].astype(np.int64) << 15) | g["b"]
    assert np.all(np.diff(key) > 0)


def test_autotune_keeps_results():
    """The launch-shape autotuner changes timings only: contacts, times and
    volumes after tuning equal those before, and the chosen shapes are among
    the candidates."""
    sc = G.scene_lattice58((6, 6, 2))
    eng = S.Stiv.for_scene(sc, pair_cap=2048, contact_cap=1 << 17)
    ds = S.DeviceScene.from_scene(sc)
    r0 = {k: (v.cpu().numpy().copy() if torch.is_tensor(v) else v) for k, v in eng.step(ds, grad=True).items()}
    choice = eng.autotune(ds)
    assert choice["best_ms"] > 0
    assert choice["narrow_ctas_per_sm"] in (0, 2, 3, 4) and choice["pieces_ctas_per_sm"] in (0, 1, 2, 3, 4)
    assert choice["fp64_blocks_per_sm"] in (0, 4, 8, 16, 32) and choice["patch_blocks_per_sm"] in (0, 2, 4, 8)
    assert choice["piece_levels"] in (0, 2, 3, 4)
    for use_graph in (False, True, True):
        r1 = eng.step(ds, grad=True, use_graph=use_graph)
        for k in ("i", "j", "shift", "pair", "type", "a", "b"):
            assert np.array_equal(r1[k].cpu().numpy(), r0[k]), k
        assert np.array_equal(bits(r1["tau"].cpu().numpy()), bits(r0["tau"]))
        assert np.array_equal(r1["V_pair"].cpu().numpy(), r0["V_pair"])
