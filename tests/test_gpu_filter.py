"""The certified FP32 rejection in the narrow phase changes no result: with
and without it (stiv_params.exact_only) the contact lists, contact times and
counts agree bit for bit, on a 144-vesicle piece of the 58% lattice workload
(p = 16 -> 32) in both precision forms and at the default and deepest
refinement of the piece test."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,levels", [(S.STIV_FP64, 2), (S.STIV_MIXED, 2), (S.STIV_FP64, 6)])
def test_filter_is_exact(precision, levels):
    sc = G.scene_lattice58((6, 6, 2))
    kw = dict(precision=precision, pair_cap=2048, contact_cap=1 << 17)
    eng_f = S.Stiv.for_scene(sc, precision=precision, pair_cap=2048, contact_cap=1 << 17)
    eng_f.set_tuning(piece_levels=levels)
    eng_x = S.Stiv.for_scene(sc, precision=precision, pair_cap=2048, contact_cap=1 << 17, exact_only=True)
    g_f = run_gpu(sc, eng=eng_f, **kw)
    g_x = run_gpu(sc, eng=eng_x, **kw)
    assert g_f["counts"][S.C_VF] + g_f["counts"][S.C_EE] > 10000
    for k in ("i", "j", "shift", "pair", "type", "a", "b"):
        assert np.array_equal(g_f[k], g_x[k]), k
    assert np.array_equal(g_f["tau"].view(np.int64), g_x["tau"].view(np.int64))
    assert np.array_equal(g_f["w"].view(np.int64), g_x["w"].view(np.int64))
    for c in (S.C_PAIRS, S.C_PRIM, S.C_VF, S.C_EE, S.C_CPAIRS, S.C_DEGEN, S.C_PATCH):
        assert g_f["counts"][c] == g_x["counts"][c], c
    # the filter removes most of the FP64 work
    assert g_f["counts"][S.C_FLOPS] < 0.5 * g_x["counts"][S.C_FLOPS]
