"""Test helpers: run the CUDA path through the C-ABI binding and bring results
to the host as numpy arrays; run the oracle (passed in) over a whole scene and
compare whole contact lists.  Test infrastructure only."""
import numpy as np
import torch

from paper_1812_04719_gb300 import stiv as S


def run_gpu(sc, precision=S.STIV_FP64, grad=True, use_graph=False, include_ee=True, pair_cap=256,
            contact_cap=4096, eng=None):
    eng = eng or S.Stiv.for_scene(sc, precision=precision, include_ee=include_ee, pair_cap=pair_cap,
                                  contact_cap=contact_cap)
    ds = S.DeviceScene.from_scene(sc, precision=precision)
    r = eng.step(ds, grad=grad, use_graph=use_graph)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    out["verts"] = ds.verts.double().cpu().numpy()
    out["eng"] = eng
    out["ds"] = ds
    return out


def run_gpu_on(sc, X, precision=S.STIV_FP64, grad=True, use_graph=False, replays=1, include_ee=True, pair_cap=256,
               contact_cap=4096, eng=None):
    """Detection, volumes (and gradient rows) on given FP64 vertices X (the
    oracle's synthesis): uploaded in the form's vertex type, the step run
    without the GPU upsampling.  out["verts"] holds the values the device
    used, widened to FP64 (the oracle's input)."""
    eng = eng or S.Stiv.for_scene(sc, precision=precision, include_ee=include_ee, pair_cap=pair_cap,
                                  contact_cap=contact_cap)
    ds = S.DeviceScene.from_scene(sc, precision=precision)
    Xd = np.ascontiguousarray(X, dtype=np.float32 if precision == S.STIV_MIXED else np.float64)
    ds.verts.copy_(torch.from_numpy(Xd))
    for _ in range(replays):
        r = eng.step(ds, grad=grad, upsample=False, use_graph=use_graph)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    out["verts"] = Xd.astype(np.float64)
    out["eng"] = eng
    out["ds"] = ds
    return out


def verts_list(sc, flat):
    """Flat vertex array -> list of [2][3][n_v] arrays (FP64)."""
    offs = sc.vert_off()
    sizes = sc.vert_sizes()
    return [flat[o:o + s].reshape(2, 3, -1).astype(np.float64) for o, s in zip(offs, sizes)]


def gpu_pairs_rows(g):
    sv = S.shift_vec(g["shift"])
    return np.concatenate([g["i"][:, None], g["j"][:, None], sv], axis=1).astype(np.int32)


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


def oracle_scene(orc, sc, flat, grad_wrt="X1"):
    Xs = verts_list(sc, flat)
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True, grad_wrt=grad_wrt)
    c["pairs"] = pairs
    return c


def assert_whole_list(g, c):
    assert g["counts"][S.C_STATUS] == 0
    assert np.array_equal(gpu_pairs_rows(g), c["pairs"])
    n = len(c["pair"])
    assert n > 500_000 and len(g["pair"]) == n
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.array_equal(bits(g["w"]), bits(c["w"]))
    assert np.all(np.abs(g["V"] - c["V"]) <= 1e-10 * np.abs(c["V"]))
    assert np.all(np.abs(g["V_pair"] - c["V_pair"]) <= 1e-10 * np.abs(c["V_pair"]))
    scale = np.abs(c["grad"]).reshape(n, -1).max(axis=1)
    err = np.abs(g["grad"] - c["grad"]).reshape(n, -1).max(axis=1)
    assert np.all(err <= 1e-9 * scale)
    assert np.array_equal(g["gves"], c["gves"]) and np.array_equal(g["gvid"], c["gvid"])
    assert g["counts"][S.C_PRIM] == c["counts"][1]
    assert g["counts"][S.C_DEGEN] == c["counts"][2]
