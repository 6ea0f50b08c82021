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


def contact_keys(i, j, shift, pair, typ, a, b, tau, skip=None):
    """Each contact as (i, j, shift, type, a, b, tau bits), leaving out those
    of vesicle `skip`."""
    tb = np.ascontiguousarray(tau, dtype=np.float64).view(np.int64)
    out = set()
    for k in range(len(pair)):
        q = int(pair[k])
        key = (int(i[q]), int(j[q]), int(shift[q]))
        if skip is not None and skip in key[:2]:
            continue
        out.add(key + (int(typ[k]), int(a[k]), int(b[k]), int(tb[k])))
    return out


@pytest.mark.parametrize("precision", [S.STIV_FP64, S.STIV_MIXED])
@pytest.mark.parametrize("bad", [0, -3, "p_max+1", 1000])
def test_bad_order_is_flagged_and_skipped(precision, bad):
    """A per-vesicle order outside [1, p_max] on the device (the host check
    bypassed): the step reports STIV_ERR_INPUT with STIV_F_BAD_ORDER alone,
    that vesicle is left out, every other pair and contact is the one of the
    valid scene bit for bit, mesh fidelity gives NaN for it, the adjoint
    leaves its coefficient block untouched, and the context stays usable."""
    from tests.test_gpu_parity import SCENES
    sc = SCENES["periodic_p3"]()
    caps = dict(pair_cap=512, contact_cap=1 << 15)
    ref = run_gpu(sc, precision=precision, grad=False, **caps)
    k = int(ref["i"][ref["pair"][0]])
    eng = S.Stiv.for_scene(sc, precision=precision, **caps)
    ds = S.DeviceScene.from_scene(sc, precision=precision)
    ds.p[k] = ds.p_max + 1 if bad == "p_max+1" else bad
    with pytest.raises(S.StivError) as e:
        eng.step(ds, grad=False)
    assert e.value.status == S.STIV_ERR_INPUT
    b = eng.buf
    counts = b.counts.cpu().numpy()
    assert counts[S.C_STATUS] == S.F_BAD_ORDER
    npair, ncon = int(counts[S.C_PAIRS]), int(counts[S.C_VF] + counts[S.C_EE])
    ci, cj, cs = (x[:npair].cpu().numpy() for x in (b.ci, b.cj, b.cs))
    assert not np.any(ci == k) and not np.any(cj == k)
    want_pairs = {(int(a_), int(b_), int(s_)) for a_, b_, s_ in zip(ref["i"], ref["j"], ref["shift"]) if k not in (a_, b_)}
    assert {(int(a_), int(b_), int(s_)) for a_, b_, s_ in zip(ci, cj, cs)} == want_pairs
    got = contact_keys(ci, cj, cs, *(x[:ncon].cpu().numpy() for x in (b.pair, b.type, b.a, b.b, b.tau)))
    want = contact_keys(ref["i"], ref["j"], ref["shift"], ref["pair"], ref["type"], ref["a"], ref["b"], ref["tau"],
                        skip=k)
    assert len(want) > 0 and got == want
    # mesh fidelity: NaN for the skipped vesicle, the valid scene's values elsewhere
    err = eng.mesh_fidelity(ds).cpu().numpy()
    err_ref = ref["eng"].mesh_fidelity(ref["ds"]).cpu().numpy()
    others = np.arange(sc.n) != k
    assert np.all(np.isnan(err[k])) and np.array_equal(err[others], err_ref[others])
    # adjoint to the coefficients: the skipped vesicle's block keeps its values
    st = torch.cuda.current_stream().cuda_stream
    gX = torch.randn(ds.verts.numel(), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    gc = torch.full_like(ds.coef, 7.0)
    gc_ref = torch.full_like(ds.coef, 7.0)
    for h, d, out in ((eng.h, ds, gc), (ref["eng"].h, ref["ds"], gc_ref)):
        S.stiv_grad_to_coef(h, st, d.n, d.p_max, S._ptr(d.p), S._ptr(d.coef_off), S._ptr(d.vert_off), S._ptr(gX),
                            S._ptr(out))
    torch.cuda.synchronize()
    gc, gc_ref = gc.cpu().numpy(), gc_ref.cpu().numpy()
    o0 = int(sc.coef_off[k])
    o1 = o0 + 6 * (int(sc.p[k]) + 1) ** 2
    assert np.all(gc[o0:o1] == 7.0)
    mask = np.ones(len(gc), dtype=bool)
    mask[o0:o1] = False
    assert np.array_equal(gc[mask], gc_ref[mask])
    # the context still runs the path
    g = run_gpu(sc, precision=precision, grad=False, **caps)
    assert g["counts"][S.C_STATUS] == 0 and np.array_equal(g["tau"].view(np.int64), ref["tau"].view(np.int64))
