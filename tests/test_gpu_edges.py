"""Edge cases on the GPU: fewer than two vesicles (no pairs can exist) and
the largest order the library accepts (p = 32, meshes of order P = 64), both
forms, against the oracle."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import gpu_pairs_rows, run_gpu, run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices

pytestmark = pytest.mark.gpu


def bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.int64)


@pytest.mark.parametrize("precision", [S.STIV_FP64, S.STIV_MIXED])
def test_one_vesicle(orc, precision):
    """A single vesicle: upsampled as the oracle does, no candidate pair, no
    contact, every count zero."""
    base = G.scene_small((2, 1, 1), p=4, seed=3)
    sc = G._pack("one", base.p[:1], [base.coef_of(0)], base.L, base.centers[:1])
    g = run_gpu(sc, precision=precision)
    assert np.all(g["counts"] == 0)
    assert len(g["i"]) == 0 and len(g["pair"]) == 0
    p = int(sc.p[0])
    Xo = orc.synth_vesicle(p, int(sc.P[0]), sc.coef_of(0))
    if precision == S.STIV_FP64:
        assert np.abs(g["verts"] - Xo.ravel()).max() <= 1e-13 * np.abs(Xo).max()
    else:
        # the MIXED synthesis bound per vertex coordinate of each field
        a1 = np.abs(sc.coef_of(0)[:, :, 1:]).sum(axis=-1)[:, :, None]
        bound = 2.0 ** -23 * np.abs(Xo) + 2.0 ** -19 * a1 * np.sqrt((2 * p + 1) / (2 * np.pi))
        assert np.all(np.abs(g["verts"].reshape(Xo.shape) - Xo) <= bound)


def test_no_vesicles():
    """n_ves = 0 through the C ABI: both calls succeed and the counts are
    zeroed."""
    sc = G.scene_small((2, 1, 1), p=4, seed=3)
    eng = S.Stiv.for_scene(sc)
    b = S.Buffers(torch.device("cuda"), 8, 8, grad=False)
    b.counts.fill_(7)
    st = torch.cuda.current_stream().cuda_stream
    cand, out = b.pairs_struct(), b.contacts_struct()
    assert S.lib().stiv_upsample(eng.h, st, 0, 1, 0, 0, 0, 0, 0) == S.STIV_OK
    rc = S.lib().stiv_detect(eng.h, st, 0, 1, 0, 0, 0, ctypes.byref(cand), ctypes.byref(out), b.counts.data_ptr())
    assert rc == S.STIV_OK
    torch.cuda.synchronize()
    assert int(b.counts.abs().sum().item()) == 0


@pytest.mark.parametrize("precision", [S.STIV_FP64, S.STIV_MIXED])
def test_largest_order(orc, precision):
    """Two vesicles at p = 32 (P = 64, 8322 vertices each: the largest mesh,
    whose triangle and edge ids and patch counts fill the descriptor fields
    closest to their limits) colliding over the step: candidate pairs,
    primitive pairs tested and contacts (keys, times and weights bit for bit)
    as the oracle's on the same vertices; V per pair within 1e-10."""
    sc = G.two_vesicles(p=32, seed=4, gap=0.02, approach=0.6)
    g = run_gpu_on(sc, oracle_vertices(sc), precision=precision, grad=False, pair_cap=16, contact_cap=1 << 18)
    Xs = verts_list(sc, g["verts"])
    boxes = np.stack([orc.vesicle_box(X, sc.d_m) for X in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    assert np.array_equal(gpu_pairs_rows(g), pairs)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=False)
    assert len(c["pair"]) > 100
    for k in ("pair", "type", "a", "b"):
        assert np.array_equal(g[k], c[k]), k
    assert np.array_equal(bits(g["tau"]), bits(c["tau"]))
    assert np.array_equal(bits(g["w"]), bits(c["w"]))
    assert g["counts"][S.C_PRIM] == c["counts"][1]
    assert np.all(np.abs(g["V_pair"] - c["V_pair"][:len(g["V_pair"])]) <= 1e-10 * np.abs(c["V_pair"][:len(g["V_pair"])]))
