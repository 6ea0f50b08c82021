"""The contact LCP on the GPU (Sec. 3.2, Eq. 3.7; Sec. 3.3.3, Alg. 3) against
the oracle: B and q formed from a step's contacts and volume gradients, and
the minimum-map Newton solution, on a small periodic suspension (p = 3 -> 6,
B with off-diagonal entries even without the translation term) and the
144-vesicle piece of the 58% lattice workload (p = 16 -> 32).  Every input of
both sides is the oracle's vertex synthesis; the oracle's B is formed from its
own contacts and dual-number gradients."""
import os

import numpy as np
import pytest
import torch

from oracle import lcp as L
from paper_1812_04719_gb300 import scenegen as G
from paper_1812_04719_gb300 import stiv as S
from tests.gpu_run import run_gpu_on, verts_list
from tests.oracle_pool import oracle_vertices

pytestmark = pytest.mark.gpu

SCENES = {
    "periodic_p3": lambda: G.scene_small((4, 4, 2), p=3, seed=6, periodic=True),
    "lattice_144_p16": lambda: G.scene_lattice58((6, 6, 2)),
}


def weights(sc, kind):
    """Per-vesicle m_i and t_i of M_ii = m_i I + t_i (1 1^T (x) I_3)."""
    if kind == "identity":
        return None, None
    rng = np.random.default_rng(17)
    m = rng.uniform(0.5, 2.0, sc.n)
    t = rng.uniform(0.5, 2.0, sc.n) / np.array([G.nverts(int(P)) for P in sc.P])
    return m, t


def oracle_lcp(orc, sc, X, m, t):
    """Rows (pairs with contacts, ascending), B by Alg. 3, q = -V, from the
    oracle's candidate pairs, contacts and gradients on the vertices X."""
    Xs = verts_list(sc, X)
    boxes = np.stack([orc.vesicle_box(x, sc.d_m) for x in Xs])
    pairs = orc.candidate_pairs(boxes, sc.L)
    c = orc.contacts(sc.P, Xs, pairs, sc.L, sc.eps * sc.dt, grad=True, nthreads=os.cpu_count() or 1)
    rows = np.unique(c["pair"])
    nverts = [G.nverts(int(P)) for P in sc.P]
    jr = L.jacobian_rows(len(rows), np.searchsorted(rows, c["pair"]), c["grad"], c["gves"], c["gvid"], nverts)
    B = L.lcp_matrix_alg3(jr, np.ones(sc.n) if m is None else m, t)
    ves = pairs[rows][:, :2]
    share = (ves[:, None, 0] == ves[None, :, 0]) | (ves[:, None, 0] == ves[None, :, 1]) | \
            (ves[:, None, 1] == ves[None, :, 0]) | (ves[:, None, 1] == ves[None, :, 1])
    return dict(rows=rows, B=B, q=-c["V_pair"][rows], share=share)


_cache = {}


def prepared(orc, name, kind):
    key = (name, kind)
    if key not in _cache:
        sc = SCENES[name]()
        X = oracle_vertices(sc)
        m, t = weights(sc, kind)
        o = oracle_lcp(orc, sc, X, m, t)
        g = run_gpu_on(sc, X, grad=True, pair_cap=2048, contact_cap=1 << 17)
        lcp = S.ContactLCP(row_cap=64, nnz_cap=256)       # grown by the wrapper
        dev = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64, device="cuda")
        A = lcp.assemble(g["eng"], g["ds"], dev(m), dev(t))
        torch.cuda.synchronize()
        a = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in A.items()}
        n = a["n"]
        Bg = np.zeros((n, n))
        for r in range(n):
            cols = a["col"][a["row_ptr"][r]:a["row_ptr"][r + 1]]
            assert np.all(np.diff(cols) > 0)
            Bg[r, cols] = a["val"][a["row_ptr"][r]:a["row_ptr"][r + 1]]
        _cache[key] = dict(sc=sc, o=o, g=g, lcp=lcp, a=a, Bg=Bg)
    return _cache[key]


@pytest.mark.parametrize("kind", ["identity", "weighted"])
@pytest.mark.parametrize("name", list(SCENES))
def test_lcp_matrix_matches_oracle(orc, name, kind):
    """Rows and their pairs exactly; q within 1e-10 (the volumes' bar); the
    sparsity pattern exactly (every pair of volumes sharing a vesicle); each
    entry within 1e-9 sqrt(B_jj B_kk) (the gradients' bar); B symmetric bit
    for bit."""
    P = prepared(orc, name, kind)
    o, a, Bg = P["o"], P["a"], P["Bg"]
    assert a["n"] == len(o["rows"]) and a["n"] >= 60
    assert np.array_equal(a["row_pair"], o["rows"].astype(np.int32))
    assert np.all(np.abs(a["q"] - o["q"]) <= 1e-10 * np.abs(o["q"]))
    pattern = np.zeros_like(o["share"])
    for r in range(a["n"]):
        pattern[r, a["col"][a["row_ptr"][r]:a["row_ptr"][r + 1]]] = True
    assert np.array_equal(pattern, o["share"])
    assert a["nnz"] == int(o["share"].sum())
    d = np.sqrt(np.outer(np.diag(o["B"]), np.diag(o["B"])))
    err = np.abs(Bg - o["B"])
    assert np.all(err <= 1e-9 * d + 1e-300), float((err / np.maximum(d, 1e-300)).max())
    assert np.array_equal(Bg, Bg.T)
    if kind == "weighted":      # the translation term couples every shared vesicle
        assert np.all((Bg != 0) == o["share"])
    print(f"{name}/{kind}: n={a['n']} nnz={a['nnz']} max err/sqrt(BjjBkk)={float((err / d).max()):.2e}")


@pytest.mark.parametrize("kind", ["identity", "weighted"])
@pytest.mark.parametrize("name", list(SCENES))
def test_lcp_solve_oracle_matrix(orc, name, kind):
    """stiv_lcp_solve on the oracle's own B and q equals the oracle's
    minimum-map Newton solution, and satisfies the complementarity conditions
    under the oracle's B."""
    P = prepared(orc, name, kind)
    o = P["o"]
    B, q = o["B"], o["q"]
    x_o, it_o, res_o = L.minmap_newton(B, q)
    assert res_o <= 1e-12
    rp = np.concatenate([[0], np.cumsum(o["share"].sum(axis=1))])
    cols = np.concatenate([np.nonzero(o["share"][r])[0] for r in range(len(q))])
    vals = np.concatenate([B[r, o["share"][r]] for r in range(len(q))])
    lcp = S.ContactLCP()
    lcp.load_csr(rp, cols, vals, q)
    res = lcp.solve(P["g"]["eng"], tol=1e-12)
    x = res["lam"].cpu().numpy()
    assert res["status"] == 0 and res["residual"] <= 1e-12, res
    assert np.all(np.abs(x - x_o) <= 1e-8 * np.abs(x_o).max())
    w = B @ x + q
    assert np.abs(np.minimum(x, w)).max() <= 1e-11 * np.abs(q).max()
    print(f"{name}/{kind}: newton {res['newton']} (oracle {it_o}), cg {res['cg']}, "
          f"max|dx|/max|x| {np.abs(x - x_o).max() / np.abs(x_o).max():.2e}")


@pytest.mark.parametrize("kind", ["identity", "weighted"])
@pytest.mark.parametrize("name", list(SCENES))
def test_lcp_end_to_end(orc, name, kind):
    """Assembly and solve both on the GPU: the multipliers equal the oracle's
    (its own B and q) within the sensitivity of the solution to B's rounding,
    and they solve the oracle's LCP to that accuracy."""
    P = prepared(orc, name, kind)
    o = P["o"]
    res = P["lcp"].solve(P["g"]["eng"], tol=1e-12)
    x = res["lam"].cpu().numpy()
    assert res["status"] == 0, res
    x_o, _, _ = L.minmap_newton(o["B"], o["q"])
    assert np.all(np.abs(x - x_o) <= 1e-7 * np.abs(x_o).max()), np.abs(x - x_o).max() / np.abs(x_o).max()
    assert np.all(x >= 0)
    w = o["B"] @ x + o["q"]
    assert np.abs(np.minimum(x, w)).max() <= 1e-8 * np.abs(o["q"]).max()
    assert (x > 0).sum() >= len(x) // 2


@pytest.mark.parametrize("n", [1, 3, 5, 8])
def test_lcp_solve_brute_force(orc, n):
    """Small dense positive definite LCPs: the unique solution found by
    enumerating all 2^n active sets."""
    rng = np.random.default_rng(100 + n)
    eng = S.Stiv()
    lcp = S.ContactLCP()
    for _ in range(10):
        Gm = rng.normal(size=(n, n))
        B = Gm @ Gm.T + 0.1 * np.eye(n)
        q = rng.normal(size=n)
        sols = L.brute_force_lcp(B, q)
        assert len(sols) == 1
        lcp.load_csr(np.arange(n + 1) * n, np.tile(np.arange(n), n), B.ravel(), q)
        res = lcp.solve(eng, tol=1e-13)
        x = res["lam"].cpu().numpy()
        assert res["status"] == 0, res
        assert np.allclose(x, sols[0], rtol=1e-9, atol=1e-12)


def test_lcp_solve_large_sparse(orc):
    """A 4000-row sparse, diagonally dominant LCP (too large for the solve's
    shared-memory staging: the vectors stay in global scratch): the oracle's
    minimum-map Newton solution."""
    rng = np.random.default_rng(7)
    n = 4000
    B = np.zeros((n, n))
    for i in range(n):
        for j in rng.choice(n, 3, replace=False):
            if j != i:
                v = rng.uniform(-0.3, 0.3)
                B[i, j] += v
                B[j, i] += v
    B += np.diag(np.abs(B).sum(axis=1) + rng.uniform(0.5, 2.0, n))
    q = rng.normal(size=n)
    x_o, _, res_o = L.minmap_newton(B, q)
    assert res_o <= 1e-12
    nz = B != 0
    rp = np.concatenate([[0], np.cumsum(nz.sum(axis=1))])
    cols = np.nonzero(nz)[1]
    lcp = S.ContactLCP()
    lcp.load_csr(rp, cols, B[nz], q)
    res = lcp.solve(S.Stiv(), tol=1e-12)
    x = res["lam"].cpu().numpy()
    assert res["status"] == 0, res
    assert np.all(np.abs(x - x_o) <= 1e-10 * np.abs(x_o).max())


def test_lcp_degenerate_cases(orc):
    """No contact volumes: an empty matrix and a solve that returns at once;
    q >= 0: lambda = 0 without a Newton step."""
    sc = G.two_vesicles(p=4, seed=1, gap=1.0, approach=0.1)
    g = run_gpu_on(sc, oracle_vertices(sc), grad=True)
    assert g["counts"][S.C_VF] + g["counts"][S.C_EE] == 0
    lcp = S.ContactLCP(row_cap=4, nnz_cap=4)
    A = lcp.assemble(g["eng"], g["ds"])
    assert A["n"] == 0 and A["nnz"] == 0
    res = lcp.solve(g["eng"])
    assert res["status"] == 0 and res["newton"] == 0
    lcp.load_csr([0, 1, 2], [0, 1], [2.0, 3.0], [0.5, 0.0])
    res = lcp.solve(g["eng"])
    assert res["status"] == 0 and res["newton"] == 0
    assert np.all(res["lam"].cpu().numpy() == 0.0)


def test_lcp_capacity_overflow(orc):
    """Too few rows or nonzeros: reported in dims[2] (not an error of the
    call), the solve refuses the matrix (status 1); the wrapper grows its
    buffers and the result then equals that of ample capacities bit for bit."""
    P = prepared(orc, "periodic_p3", "weighted")
    g = P["g"]
    m, t = weights(P["sc"], "weighted")
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    for rcap, zcap, flag in ((8, 4096, 1), (4096, 16, 2)):
        lcp = S.ContactLCP(row_cap=rcap, nnz_cap=zcap)
        b = g["eng"].buf
        st = lcp.struct()
        rc = S.lib().stiv_lcp_matrix(g["eng"].h, 0, g["ds"].n, g["ds"].p_max, b.pairs_struct(), b.contacts_struct(),
                                     b.counts.data_ptr(), b.Vp.data_ptr(), b.grad.data_ptr(), b.gves.data_ptr(),
                                     b.gvid.data_ptr(), dev(m).data_ptr(), dev(t).data_ptr(), st)
        assert rc == S.STIV_OK
        torch.cuda.synchronize()
        dims = lcp.dims.cpu().numpy()
        assert dims[2] & flag
        assert dims[0] <= rcap
        res = lcp.solve(g["eng"])
        assert res["status"] == 1
    lcp = S.ContactLCP(row_cap=8, nnz_cap=16)
    A = lcp.assemble(g["eng"], g["ds"], dev(m), dev(t))
    a = P["a"]
    assert A["n"] == a["n"] and A["nnz"] == a["nnz"]
    assert np.array_equal(A["col"].cpu().numpy(), a["col"])
    assert np.array_equal(A["val"].cpu().numpy().view(np.int64), a["val"].view(np.int64))


def test_lcp_deterministic(orc):
    """Assembling twice gives the same bits (every sum in a fixed order)."""
    P = prepared(orc, "lattice_144_p16", "weighted")
    m, t = weights(P["sc"], "weighted")
    dev = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    lcp = S.ContactLCP(row_cap=P["lcp"].row_cap, nnz_cap=P["lcp"].nnz_cap)
    A = lcp.assemble(P["g"]["eng"], P["g"]["ds"], dev(m), dev(t))
    assert np.array_equal(A["val"].cpu().numpy().view(np.int64), P["a"]["val"].view(np.int64))
    assert np.array_equal(A["q"].cpu().numpy().view(np.int64), P["a"]["q"].view(np.int64))
