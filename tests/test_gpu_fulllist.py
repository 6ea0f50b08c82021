"""Whole-list parity on the benchmark's workload: 1440 prolate vesicles at 58%
volume fraction on the staggered lattice, p = 16 -> 32, in the launch
configuration the benchmark times (autotuned launch shapes, CUDA-graph
replay of the whole step).

- FP64 form, on the oracle's own FP64 synthesis: every candidate pair, every
  contact (pair, type, primitive ids; contact time and inside-test weights
  bit for bit), V per contact and per pair within 1e-10 relative, every
  gradient row within 1e-9 of its row's largest entry, against the oracle's
  all-pairs Alg. 2 over the whole scene (Eq. 3.1, Eq. 3.2, Alg. 2
  checkContact).
- MIXED form end to end: the tensor-core synthesis writes the FP32
  vertices, and the oracle recomputes the whole scene on exactly those
  vertices (widened to FP64), with the same bars.
- The certified FP32 rejection stages are checked against the exact path
  (stiv_params.exact_only = 1: every exact-box pair through the FP64 test)
  at this size, in both forms, GPU against GPU.
- The MIXED form end to end against the FP64 oracle on the oracle's own
  synthesis: the stated accuracy bounds of the precision form
  (paper_1812_04719_gb300/accuracy.py) on V, the contact lists and the
  gradient rows.

The oracle runs each whole scene on the host cores (about a minute on 16
cores per form)."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import accuracy as A
from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import assert_whole_list, oracle_scene
from tests.oracle_pool import oracle_vertices

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


@pytest.fixture(scope="module")
def scene():
    sc = G.scene_1440()
    return sc, oracle_vertices(sc)


def bench_engine(sc, prec, exact_only=False):
    """An engine set up as the benchmark sets it up: buffers sized by a first
    step, launch shapes picked by the autotuner."""
    eng = S.Stiv.for_scene(sc, precision=prec, pair_cap=8192, contact_cap=1 << 20, exact_only=exact_only)
    ds = S.DeviceScene.from_scene(sc, precision=prec)
    eng.step(ds, grad=True)
    eng.autotune(ds)
    return eng, ds


def replay(eng, ds, upsample, replays=3):
    """Graph replays of the whole step; the last one's outputs on the host."""
    for _ in range(replays):
        r = eng.step(ds, grad=True, upsample=upsample, use_graph=True)
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    out["verts"] = ds.verts.double().cpu().numpy()
    return out


@pytest.fixture(scope="module")
def fp64_run(scene):
    sc, Xo = scene
    eng, ds = bench_engine(sc, S.STIV_FP64)
    ds.verts.copy_(torch.from_numpy(Xo))
    g = replay(eng, ds, upsample=False)
    eng.close()
    return g


@pytest.fixture(scope="module")
def oracle_fp64(orc, scene):
    sc, Xo = scene
    return oracle_scene(orc, sc, Xo)


def test_fp64_form_whole_list(fp64_run, oracle_fp64):
    assert_whole_list(fp64_run, oracle_fp64)


@pytest.fixture(scope="module")
def mixed_run(scene):
    sc, _ = scene
    eng, ds = bench_engine(sc, S.STIV_MIXED)
    g = replay(eng, ds, upsample=True)           # the tensor-core synthesis writes the vertices
    g["grad_x0"] = eng.grad_x0(ds).cpu().numpy()
    eng.close()
    return g


def test_mixed_form_whole_list_end_to_end(orc, scene, mixed_run):
    sc, _ = scene
    c = oracle_scene(orc, sc, mixed_run["verts"])
    assert_whole_list(mixed_run, c)


@pytest.mark.parametrize("prec", [S.STIV_FP64, S.STIV_MIXED], ids=["fp64", "mixed"])
def test_filter_cascade_equals_exact_path(scene, prec):
    """The certified FP32 stages (Bernstein certificate, piece test) change
    nothing: the filtered step and the exact step (every exact-box pair
    through the FP64 contact test) give the same lists bit for bit."""
    sc, Xo = scene
    Xd = torch.from_numpy(np.ascontiguousarray(Xo, dtype=np.float32 if prec == S.STIV_MIXED else np.float64))
    runs = []
    for exact in (False, True):
        eng, ds = bench_engine(sc, prec, exact_only=exact)
        ds.verts.copy_(Xd)
        runs.append(replay(eng, ds, upsample=False, replays=2))
        eng.close()
    f, e = runs
    assert e["counts"][S.C_EXACT] == e["counts"][S.C_PRIM] > f["counts"][S.C_EXACT]
    for k in ("i", "j", "shift", "pair", "type", "a", "b", "gves", "gvid"):
        assert np.array_equal(f[k], e[k]), k
    for k in ("tau", "w", "V", "V_pair", "grad"):
        assert np.array_equal(bits(f[k]), bits(e[k])), k


@pytest.fixture(scope="module")
def oracle_fp64_x0(orc, scene):
    sc, Xo = scene
    return oracle_scene(orc, sc, Xo, grad_wrt="X0")


def test_mixed_form_accuracy_bounds(scene, mixed_run, oracle_fp64, oracle_fp64_x0):
    """The precision form end to end (tensor-core synthesis, FP32 vertices,
    FP64 detection and volumes) against the FP64 oracle on its own synthesis:
    (1) |dV_k| <= S_k delta_k for every contact in both lists; (2) every
    contact in one list only has decision margins below 4 delta_k; (3) every
    gradient row of a contact in both lists within 4 kappa_k of its largest
    entry; (4) every vesicle pair's V within the sum of its contacts' bounds
    and of its one-list contacts' volumes.  Almost every contact is in both
    lists."""
    sc, Xo = scene
    c = oracle_fp64
    rb = dict(c)
    pr = c["pairs"]
    rb["i"], rb["j"] = pr[:, 0], pr[:, 1]
    rb["shift"] = 9 * (pr[:, 2] + 1) + 3 * (pr[:, 3] + 1) + (pr[:, 4] + 1)
    assert np.array_equal(oracle_fp64_x0["pair"], c["pair"]) and np.array_equal(oracle_fp64_x0["a"], c["a"])
    pdelta = A.point_delta(sc.p, sc.coef_of, sc.vert_off(), Xo)
    res = A.compare(mixed_run, mixed_run["verts"], rb, Xo, oracle_fp64_x0["grad"], pdelta, sc.vert_off(), sc.L)
    print({k: v for k, v in res.items()})
    assert res["contacts_both"] >= 0.999 * res["contacts_fp64"]
    assert res["bound1_V_holds"], res["V_ratio_max"]
    assert res["bound2_lists_hold"], res["symdiff_margin_max"]
    assert res["bound3_grad_holds"], res["grad_ratio_max"]
    assert res["bound4_pairs_hold"], res["pairs_exceeding_bound"]
