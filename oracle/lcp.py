"""Plain FP64 CPU oracle of the contact LCP (Sec. 3.2, Eq. 3.7; Sec. 3.3.3,
Alg. 3).  TEST INFRASTRUCTURE ONLY: only the test suite may import it; the
CUDA product path never imports or calls it, and it shares no code with it.

Each contact-resolving step solves the linear complementarity problem

    0 <= V + B lambda   perp   lambda >= 0,        B = J M J^T,

with one row per contact volume (here: per interfering vesicle pair, the sum
of its contacts' volumes), J the Jacobian of the volumes with respect to the
end-of-step positions X1 and M = A^-1 G the block-diagonal operator of the
locally implicit scheme (one block per vesicle).  The paper writes the
interference volume as negative (V >= 0 is the constraint); the volumes of
this code are non-negative for interference, so its LCP reads
0 <= -V + B lambda perp lambda >= 0 with the same B (the sign of J cancels).
M here is a stand-in with the block structure of A^-1 G: per vesicle i,
M_ii = m_i I + t_i (1 1^T (x) I_3), a local part plus a rigid translation of
the whole vesicle (a force at one point moves every point), so that B(j, k)
is nonzero whenever volumes j and k involve a common vesicle.
"""
from __future__ import annotations

import itertools

import numpy as np


def jacobian_rows(n_rows, row_of_contact, grad, gves, gvid, nverts):
    """Per contact volume r: {vesicle: dense [n_v][3] gradient block} summed
    over the contacts of r (grad [k][4][3], point k,q at vertex gvid of
    vesicle gves)."""
    rows = [dict() for _ in range(n_rows)]
    for k in range(len(row_of_contact)):
        r = row_of_contact[k]
        for q in range(4):
            v = int(gves[k, q])
            blk = rows[r].get(v)
            if blk is None:
                blk = np.zeros((nverts[v], 3))
                rows[r][v] = blk
            blk[gvid[k, q]] += grad[k, q]
    return rows


def lcp_matrix_alg3(rows, m_ves, t_ves=None):
    """Alg. 3: for each vesicle i, for each pair (j, k) of contact volumes that
    involve i, B(j, k) += g_j . M_ii g_k with g the Jacobian rows restricted to
    the sample points of vesicle i; with M_ii = m_i I + t_i (1 1^T (x) I_3)
    that is m_i sum_points g_j . g_k + t_i (sum_points g_j) . (sum_points g_k)."""
    n = len(rows)
    B = np.zeros((n, n))
    involved = {}
    for r, blocks in enumerate(rows):
        for v in blocks:
            involved.setdefault(v, []).append(r)
    for i in sorted(involved):
        for j in involved[i]:
            gj = rows[j][i]
            for k in involved[i]:
                gk = rows[k][i]
                B[j, k] += m_ves[i] * float(np.sum(gj * gk))
                if t_ves is not None:
                    B[j, k] += t_ves[i] * float(gj.sum(axis=0) @ gk.sum(axis=0))
    return B


def dense_jacobian(rows, nverts):
    """J as a dense matrix over all sample points (3 columns per vertex)."""
    offs = np.concatenate([[0], np.cumsum([3 * nv for nv in nverts])])
    J = np.zeros((len(rows), int(offs[-1])))
    for r, blocks in enumerate(rows):
        for v, blk in blocks.items():
            J[r, offs[v]:offs[v + 1]] = blk.ravel()
    return J, offs


def minmap_newton(B, q, tol=1e-12, max_newton=100, max_halvings=40, alpha=1e-4):
    """Minimum-map Newton method for 0 <= B x + q perp x >= 0:
    Phi(x) = min(x, B x + q); at each step the generalised Jacobian takes the
    row of B where (B x + q)_i < x_i (active set A) and the identity row
    elsewhere; the Newton system gives dx_i = -x_i off A and
    B_AA dx_A = -(B x + q)_A - B_{A,F} dx_F on A; an Armijo line search on
    psi = |Phi|^2 / 2 along x + t dx sets the step (the Newton direction is a
    descent direction of psi; a projection onto x >= 0 inside the search can
    stall it, and at the solution min(x, w) = 0 gives x >= 0 anyway).
    Returns (x, iterations, max |Phi|)."""
    n = len(q)
    x = np.zeros(n)
    it = 0
    for it in range(max_newton + 1):
        w = B @ x + q
        phi = np.minimum(x, w)
        res = float(np.abs(phi).max()) if n else 0.0
        if res <= tol or it == max_newton:
            break
        act = w < x
        dx = -x.copy()
        if act.any():
            free = ~act
            rhs = -w[act] - B[np.ix_(act, free)] @ dx[free]
            dx[act] = np.linalg.solve(B[np.ix_(act, act)], rhs)
        psi = 0.5 * float(phi @ phi)
        t = 1.0
        for _ in range(max_halvings):
            xn = x + t * dx
            pn = np.minimum(xn, B @ xn + q)
            if 0.5 * float(pn @ pn) <= (1.0 - 2.0 * alpha * t) * psi:
                break
            t *= 0.5
        x = xn
    return x, it, res


def brute_force_lcp(B, q):
    """Every solution of the LCP by enumeration of the 2^n active sets (n <= 10):
    x_A = -B_AA^-1 q_A >= 0, x elsewhere 0, w = B x + q >= 0 off A."""
    n = len(q)
    sols = []
    for mask in itertools.product([False, True], repeat=n):
        act = np.array(mask, dtype=bool)
        x = np.zeros(n)
        if act.any():
            try:
                x[act] = np.linalg.solve(B[np.ix_(act, act)], -q[act])
            except np.linalg.LinAlgError:
                continue
        w = B @ x + q
        if np.all(x >= -1e-12) and np.all(w[~act] >= -1e-12):
            sols.append(x)
    return sols
