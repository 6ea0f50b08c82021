"""Failure detection without a GPU fault: capacity overflows are flagged and
the binding re-runs with larger buffers; non-finite input and a periodic box
too small for the image convention are flagged as input errors; a bounded
device wait gives up by itself and leaves the context usable."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import run_gpu

pytestmark = pytest.mark.gpu


def test_capacity_overflow_grows_and_matches():
    sc = G.scene_small((2, 2, 1), p=4, seed=3)
    big = run_gpu(sc, pair_cap=4096, contact_cap=1 << 16)
    small = run_gpu(sc, pair_cap=2, contact_cap=8)       # overflows, then grows
    assert small["eng"].pair_cap > 2 and small["eng"].contact_cap > 8
    for k in ("i", "j", "shift", "pair", "type", "a", "b"):
        assert np.array_equal(small[k], big[k]), k
    assert np.array_equal(small["tau"].view(np.int64), big["tau"].view(np.int64))


def test_nonfinite_input_is_flagged():
    sc = G.scene_small((2, 1, 1), p=4, seed=3)
    sc.coef = sc.coef.copy()
    sc.coef[5] = np.nan
    eng = S.Stiv.for_scene(sc, pair_cap=64, contact_cap=4096)
    ds = S.DeviceScene.from_scene(sc)
    with pytest.raises(S.StivError) as e:
        eng.step(ds, grad=False)
    assert e.value.status == S.STIV_ERR_INPUT
    counts = eng.buf.counts.cpu().numpy()
    assert counts[S.C_STATUS] & S.F_NONFINITE


def test_periodic_box_too_small_is_flagged():
    sc = G.scene_small((2, 1, 1), p=4, seed=3)
    sc.L = np.array([4.0, 4.0, 4.0])      # vesicle boxes span more than half of it
    eng = S.Stiv.for_scene(sc, pair_cap=64, contact_cap=4096)
    ds = S.DeviceScene.from_scene(sc)
    with pytest.raises(S.StivError) as e:
        eng.step(ds, grad=False)
    assert e.value.status == S.STIV_ERR_INPUT
    assert eng.buf.counts.cpu().numpy()[S.C_STATUS] & S.F_BOX_TOO_SMALL


def test_bounded_wait_gives_up_and_context_stays_usable():
    st = torch.cuda.current_stream().cuda_stream
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    S._check(S.lib().stiv_wait_selftest(st, 2_000_000, status.data_ptr()), "stiv_wait_selftest")
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    with pytest.raises(S.StivError):
        S._check(S.lib().stiv_wait_selftest(st, -1, status.data_ptr()), "stiv_wait_selftest")
    # the context still runs the path
    g = run_gpu(G.scene_small((2, 1, 1), p=4, seed=3))
    assert g["counts"][S.C_STATUS] == 0
