"""Mesh fidelity on the GPU (Sec. 3.1.2, Fig. 6) against the oracle: per
vesicle and time level, the largest distance between the order-2p triangle
mesh (as the library upsampled it) and the smooth order-p surface on the
order-(factor 2p) grid.  The oracle evaluates the series and reads the mesh
of its own synthesis."""
import numpy as np
import pytest
import torch

from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.test_gpu_parity import SCENES

pytestmark = pytest.mark.gpu


def oracle_errors(orc, sc, ves, factor):
    out = np.zeros((len(ves), 2))
    for k, v in enumerate(ves):
        p, P = int(sc.p[v]), int(sc.P[v])
        c = sc.coef_of(v)
        X = orc.synth_vesicle(p, P, c)
        for t in range(2):
            out[k, t] = orc.mesh_fidelity(p, P, c[t], X[t], factor)
    return out


def gpu_errors(sc, precision, factor):
    eng = S.Stiv.for_scene(sc, precision=precision)
    ds = S.DeviceScene.from_scene(sc, precision=precision)
    eng.upsample(ds)
    err = eng.mesh_fidelity(ds, factor=factor)
    torch.cuda.synchronize()
    return err.cpu().numpy(), float(ds.verts.abs().max().item())


CASES = [("pair_p8", 4), ("cluster_p4", 4), ("uneven_p234", 4), ("uneven_p234", 1), ("periodic_p3", 8),
         ("lattice_144_p16", 4)]


@pytest.mark.parametrize("name,factor", CASES)
def test_fidelity_fp64_matches_oracle(orc, name, factor):
    sc = G.scene_lattice58((6, 6, 2)) if name == "lattice_144_p16" else SCENES[name]()
    got, scale = gpu_errors(sc, S.STIV_FP64, factor)
    ves = list(range(sc.n)) if sc.n <= 16 else list(np.random.default_rng(1).choice(sc.n, 6, replace=False))
    ref = oracle_errors(orc, sc, ves, factor)
    if factor == 1:   # the estimate's grid is the mesh's own: the mesh passes through the series there
        assert got.max() <= 1e-13 * scale and ref.max() <= 1e-13 * scale
    else:
        assert np.all(ref > 1e-6 * scale)
    assert np.abs(got[ves] - ref).max() <= 1e-11 * scale, np.abs(got[ves] - ref).max()
    print(f"{name} x{factor}: max err {got.max():.3e}, max |gpu - oracle| {np.abs(got[ves] - ref).max():.2e}")


def test_fidelity_mixed_form(orc):
    """MIXED: the mesh is the FP32 tensor-core synthesis; the estimate differs
    from the oracle's by at most the synthesis error bound (4e-7 of the
    largest coordinate)."""
    sc = G.scene_lattice58((6, 6, 2))
    got, scale = gpu_errors(sc, S.STIV_MIXED, 4)
    ves = [0, 17, 101]
    ref = oracle_errors(orc, sc, ves, 4)
    assert np.abs(got[ves] - ref).max() <= 4e-7 * scale


def test_fidelity_second_order_on_gpu():
    """Doubling the SH order of a scene's grid (the same shapes zero-padded to
    order 2p, so the mesh order doubles) cuts the estimate by about 4."""
    sc = SCENES["pair_p8"]()
    e1, _ = gpu_errors(sc, S.STIV_FP64, 4)
    coefs = []
    for v in range(sc.n):
        c = sc.coef_of(v)
        p = int(sc.p[v])
        out = np.zeros((2, 3, (2 * p + 1) ** 2))
        out[:, :, :(p + 1) ** 2] = c
        coefs.append(out)
    sc2 = G._pack("pair_padded", np.array([2 * int(x) for x in sc.p]), coefs, sc.L, sc.centers)
    e2, _ = gpu_errors(sc2, S.STIV_FP64, 4)
    r = e1 / e2
    assert np.all((r > 3.0) & (r < 4.6)), r


def test_fidelity_arguments():
    sc = SCENES["cluster_p4"]()
    eng = S.Stiv.for_scene(sc)
    ds = S.DeviceScene.from_scene(sc)
    eng.upsample(ds)
    for bad in (0, 9):
        with pytest.raises(S.StivError):
            eng.mesh_fidelity(ds, factor=bad)
