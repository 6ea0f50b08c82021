"""The literal-reading variants on the GPU against the oracle: U_k in Eq. 3.2
as the contact point's absolute velocity, the VF-only volume (no edge-edge
contacts) and the gradient with respect to X0.  Inputs: the oracle's vertex
synthesis on both sides."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import gpu_pairs_rows, run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices
from tests.test_gpu_parity import SCENES

pytestmark = pytest.mark.gpu

NAMES = ["cluster_p4", "periodic_p3", "uneven_p234"]


def oracle_run(orc, sc, g, **kw):
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    return orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, **kw)


def rows_close(a, b, tol):
    scale = np.abs(b).reshape(len(b), -1).max(axis=1)
    err = np.abs(a - b).reshape(len(b), -1).max(axis=1)
    return np.all(err <= tol * scale + 1e-300), float((err / np.maximum(scale, 1e-300)).max())


@pytest.mark.parametrize("name", NAMES)
def test_absolute_velocity(orc, name):
    sc = SCENES[name]()
    eng = S.Stiv.for_scene(sc, pair_cap=256, contact_cap=4096, velocity=S.STIV_VEL_ABSOLUTE)
    g = run_gpu_on(sc, oracle_vertices(sc), eng=eng)
    c = oracle_run(orc, sc, g, velocity="absolute")
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.all(np.abs(g["V"] - c["V"]) <= 1e-10 * np.abs(c["V"]))
    assert np.all(np.abs(g["V_pair"] - c["V_pair"]) <= 1e-10 * np.abs(c["V_pair"]) + 1e-300)
    ok, worst = rows_close(g["grad"], c["grad"], 1e-9)
    assert ok, worst
    # the readings differ on the same contacts
    r = run_gpu_on(sc, oracle_vertices(sc))
    assert np.array_equal(r["tau"].view(np.int64), g["tau"].view(np.int64))
    assert np.any(np.abs(r["V"] - g["V"]) > 1e-6 * r["V"])


@pytest.mark.parametrize("vel", [S.STIV_VEL_RELATIVE, S.STIV_VEL_ABSOLUTE])
@pytest.mark.parametrize("name", NAMES)
def test_grad_x0(orc, name, vel):
    """dV/dX0 rows against the oracle's dual numbers seeded on X0; with the
    X1 rows they sum to zero over each contact's points."""
    sc = SCENES[name]()
    eng = S.Stiv.for_scene(sc, pair_cap=256, contact_cap=4096, velocity=vel)
    g = run_gpu_on(sc, oracle_vertices(sc), eng=eng)
    g0 = eng.grad_x0(g["ds"]).cpu().numpy()
    torch.cuda.synchronize()
    c = oracle_run(orc, sc, g, grad_wrt="X0", velocity="absolute" if vel == S.STIV_VEL_ABSOLUTE else "relative")
    assert len(g0) == len(c["pair"]) > 0
    ok, worst = rows_close(g0, c["grad"], 1e-9)
    assert ok, worst
    s = (g0 + g["grad"]).sum(axis=1)
    assert np.abs(s).max() <= 1e-9 * np.abs(g["grad"]).max()


@pytest.mark.parametrize("name", NAMES)
def test_vf_only_volume(orc, name):
    """include_ee = 0: only vertex-triangle contacts, lists bit for bit and
    volumes as the oracle's VF-only run."""
    sc = SCENES[name]()
    g = run_gpu_on(sc, oracle_vertices(sc), include_ee=False)
    c = oracle_run(orc, sc, g, include_ee=False)
    assert len(c["pair"]) > 0 and np.all(c["type"] < 2) and np.all(g["type"] < 2)
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(g["tau"].view(np.int64), c["tau"].view(np.int64))
    assert np.all(np.abs(g["V_pair"] - c["V_pair"]) <= 1e-10 * np.abs(c["V_pair"]) + 1e-300)
    assert g["counts"][S.C_EE] == 0
