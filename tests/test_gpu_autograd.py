"""Differentiation workload: 256 vesicles at 50% volume fraction, p = 12 -> 24,
FP64.  The autograd backward of the total interference volume with respect to
the SH coefficients (recomputing meshes and contacts) is checked against the
oracle's gradient (forward-mode dual numbers, then the transpose of its
synthesis) and against central finite differences with h = 1e-6."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import autograd as A
from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import verts_list
from tests.oracle_pool import oracle_vertices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c5():
    sc = G.scene_256()
    eng = S.Stiv.for_scene(sc, pair_cap=2048, contact_cap=1 << 18)
    ds = S.DeviceScene.from_scene(sc)
    coef = ds.coef.clone().requires_grad_(True)
    total = A.stiv_sum(coef, eng, ds)
    total.backward()
    torch.cuda.synchronize()
    base = eng.step(ds, grad=False)
    keys = {k: base[k].cpu().numpy().copy() for k in ("pair", "type", "a", "b")}
    return dict(sc=sc, eng=eng, ds=ds, total=float(total.item()), grad=coef.grad.detach().cpu().numpy(),
                keys=keys, counts=base["counts"].copy(), verts=ds.verts.cpu().numpy())


def test_scene_has_contacts(c5):
    assert c5["counts"][S.C_CPAIRS] > 100
    assert c5["total"] > 0


def test_gradient_matches_oracle(orc, c5):
    sc, g = c5["sc"], c5["grad"]
    Xs = verts_list(sc, oracle_vertices(sc))      # the oracle's own synthesis
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True)
    assert len(c["pair"]) == len(c5["keys"]["pair"])
    assert abs(c["V_pair"].sum() - c5["total"]) <= 1e-10 * c5["total"]
    # dense dSum/dX1 per vesicle, then the transpose of the oracle's synthesis
    gX = [np.zeros((3, G.nverts(int(P)))) for P in sc.P]
    for k in range(len(c["pair"])):
        for q in range(4):
            gX[c["gves"][k, q]][:, c["gvid"][k, q]] += c["grad"][k, q]
    err = scale = 0.0
    for v in range(sc.n):
        p, P = int(sc.p[v]), int(sc.P[v])
        got = g[sc.coef_off[v]:sc.coef_off[v] + 6 * (p + 1) ** 2].reshape(2, 3, -1)
        assert np.all(got[0] == 0)                      # X0 is a constant of the step
        ref = np.stack([orc.synth_adjoint(p, P, gX[v][d]) for d in range(3)])
        err = max(err, np.abs(got[1] - ref).max())
        scale = max(scale, np.abs(ref).max())
    assert scale > 0 and err <= 1e-9 * scale, (err, scale)


def test_gradient_central_differences(c5):
    """Central differences of the total volume on coefficients of vesicles in
    contact; a coefficient whose +-h perturbation changes the contact list is
    skipped (the volume is only piecewise smooth)."""
    sc, eng, ds, g = c5["sc"], c5["eng"], c5["ds"], c5["grad"]
    h = 1e-6
    rng = np.random.default_rng(5)
    ves = np.unique(c5["eng"].buf.ci[:c5["counts"][S.C_PAIRS]].cpu().numpy()[
        (c5["eng"].buf.Vp[:c5["counts"][S.C_PAIRS]] > 0).cpu().numpy()])
    checked = 0
    for _ in range(40):
        v = int(rng.choice(ves))
        p = int(sc.p[v])
        d = int(rng.integers(0, 3))
        n = int(rng.integers(0, min(p, 4) + 1))
        m = int(rng.integers(-n, n + 1))
        idx = int(sc.coef_off[v]) + 3 * (p + 1) ** 2 + d * (p + 1) ** 2 + n * n + n + m
        vals, same = [], True
        for sgn in (1.0, -1.0):
            coef = ds.coef.clone()
            coef[idx] += sgn * h
            with torch.no_grad():
                vals.append(float(A.stiv_sum(coef, eng, ds).item()))
            r = eng.step(S.DeviceScene(**{**ds.__dict__, "coef": coef}), grad=False)
            for k in ("pair", "type", "a", "b"):
                same = same and np.array_equal(r[k].cpu().numpy(), c5["keys"][k])
        if not same:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(g[idx]), 1e-3 * np.abs(g).max()), (idx, fd, g[idx])
        checked += 1
        if checked == 12:
            break
    assert checked >= 8
