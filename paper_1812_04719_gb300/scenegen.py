"""Seeded synthetic scenes: vesicles as spherical-harmonic (SH) coefficients at
the start (X0) and end (X1) of one time step.

This module only builds inputs.  It holds none of the method's arithmetic
(no synthesis, no boxes, no contact tests): both the CUDA path and the CPU
oracle read the same arrays it returns.

Shapes follow the paper's workloads (arXiv 1812.04719): prolate vesicles of
reduced volume 0.91 and effective radius R0 = 1.34 (Sec. 4.3), SH order p
upsampled to 2p for contact detection, dense suspensions up to 58% volume
fraction (Fig. 1, Sec. 4.3), staggered lattices (Sec. 4.5, Fig. 12).

Coefficient convention (the input format of the library): real orthonormal
SH Y_n^m without Condon-Shortley phase, index n^2 + n + m, m > 0 ~ cos(m phi),
m < 0 ~ sin(|m| phi).  In it an ellipsoid c + M (sin t cos f, sin t sin f, cos t)
has degree-0 coefficient sqrt(4 pi) c and degree-1 coefficients
sqrt(4 pi / 3) M[:, (x, y, z)] at m = (1, -1, 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R0_PAPER = 1.34          # effective radius (Sec. 4.3)
REDUCED_VOLUME = 0.91    # Sec. 4.3 / Fig. 1


def ncoef(p: int) -> int:
    return (p + 1) * (p + 1)


def nverts(P: int) -> int:
    """Vertices of the order-P mesh: (P+1) rings of 2P points plus 2 poles."""
    return 2 * P * (P + 1) + 2


def prolate_axes(reduced_volume: float = REDUCED_VOLUME, R0: float = R0_PAPER):
    """Semi-axes (a, b, b) of a prolate spheroid with the given reduced volume
    V / (4 pi R0^3 / 3), R0 = sqrt(area / 4 pi)."""
    def nu(k):  # aspect a/b = k, b = 1
        a, b = k, 1.0
        e = math.sqrt(1.0 - (b / a) ** 2)
        area = 2 * math.pi * b * b * (1 + a / (b * e) * math.asin(e))
        vol = 4.0 / 3.0 * math.pi * a * b * b
        r0 = math.sqrt(area / (4 * math.pi))
        return vol / (4.0 / 3.0 * math.pi * r0 ** 3), r0
    lo, hi = 1.0 + 1e-9, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if nu(mid)[0] > reduced_volume:
            lo = mid
        else:
            hi = mid
    k = 0.5 * (lo + hi)
    r0 = nu(k)[1]
    s = R0 / r0
    return k * s, s


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (unit quaternion, Shoemake)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2), math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3), math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    return quat_to_matrix(q)


def quat_to_matrix(q) -> np.ndarray:
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def axis_angle(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle
    return quat_to_matrix(np.concatenate([axis * math.sin(h), [math.cos(h)]]))


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def ellipsoid_coef(p: int, center, M) -> np.ndarray:
    """[3][(p+1)^2] coefficients of x = center + M u, u on the unit sphere."""
    c = np.zeros((3, ncoef(p)))
    M = np.asarray(M, dtype=np.float64)
    s0 = math.sqrt(4 * math.pi)
    s1 = math.sqrt(4 * math.pi / 3)
    for k in range(3):
        c[k, 0] = s0 * center[k]
        if p >= 1:
            c[k, 1 * 1 + 1 + 1] = s1 * M[k, 0]   # m = +1 ~ sin t cos f = u_x
            c[k, 1 * 1 + 1 - 1] = s1 * M[k, 1]   # m = -1 ~ sin t sin f = u_y
            c[k, 1 * 1 + 1 + 0] = s1 * M[k, 2]   # m = 0  ~ cos t       = u_z
    return c


def perturbation(rng: np.random.Generator, p: int, amp: float, R0: float = R0_PAPER) -> np.ndarray:
    """[3][(p+1)^2] random coefficients for 2 <= n <= p, iid U(-1,1) amp R0/(n+1)^2."""
    c = np.zeros((3, ncoef(p)))
    for n in range(2, p + 1):
        sl = slice(n * n, (n + 1) * (n + 1))
        c[:, sl] = rng.uniform(-1.0, 1.0, size=(3, 2 * n + 1)) * amp * R0 / (n + 1) ** 2
    return c


def rigid_motion(coef: np.ndarray, R: np.ndarray, t, pivot) -> np.ndarray:
    """Coefficients of x -> pivot + R (x - pivot) + t (acts on the coordinates,
    so every (n, m) column mixes across x, y, z)."""
    out = R @ coef
    shift = np.asarray(pivot) - R @ np.asarray(pivot) + np.asarray(t)
    out[:, 0] += math.sqrt(4 * math.pi) * shift
    return out


# --- Perram-Wertheim overlap test of two ellipsoids (placement only) --------

def pw_overlap(c1, A1, c2, A2, nlam: int = 65) -> bool:
    """True if ellipsoids {x : (x-c)^T A^-1 (x-c) <= 1} overlap (max_lambda F < 1)."""
    r = np.asarray(c2, dtype=np.float64) - np.asarray(c1, dtype=np.float64)
    lam = np.linspace(0.0, 1.0, nlam)[1:-1]
    best = 0.0
    for it in range(3):
        C = (1 - lam)[:, None, None] * A1[None] + lam[:, None, None] * A2[None]
        y = np.linalg.solve(C, np.broadcast_to(r, (len(lam), 3))[..., None])[..., 0]
        F = lam * (1 - lam) * (y @ r)
        k = int(np.argmax(F))
        best = max(best, float(F[k]))
        if best >= 1.0:
            return False
        lo = lam[max(k - 1, 0)]
        hi = lam[min(k + 1, len(lam) - 1)]
        lam = np.linspace(lo, hi, 17)
    return best < 1.0


def shape_matrix(R, axes) -> np.ndarray:
    M = R @ np.diag(axes)
    return M @ M.T


def min_image(d, L):
    d = np.array(d, dtype=np.float64)
    for k in range(3):
        if L[k] > 0:
            d[k] -= L[k] * np.round(d[k] / L[k])
    return d


# --- scenes -------------------------------------------------------------------

@dataclass
class Scene:
    name: str
    p: np.ndarray                 # int32 [N] SH order of each vesicle (mesh order 2p)
    coef: np.ndarray              # float64 flat: per vesicle [2 time][3][(p+1)^2]
    coef_off: np.ndarray          # int64 [N] offsets into coef
    L: np.ndarray                 # float64 [3] periodic lengths (0 = free axis)
    centers: np.ndarray           # float64 [N][3] (start of step)
    eps: float = 1.0              # epsilon of the space-time metric (App. A)
    dt: float = 0.1               # time step (Sec. 4.3)
    d_m: float = 0.0              # separation distance (cubic path: 0)
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.p.shape[0])

    @property
    def P(self) -> np.ndarray:
        return (2 * self.p).astype(np.int32)

    def vert_sizes(self) -> np.ndarray:
        return np.array([6 * nverts(int(P)) for P in self.P], dtype=np.int64)

    def vert_off(self) -> np.ndarray:
        s = self.vert_sizes()
        return np.concatenate([[0], np.cumsum(s)[:-1]]).astype(np.int64)

    def n_vert_values(self) -> int:
        return int(self.vert_sizes().sum())

    def coef_of(self, v: int) -> np.ndarray:
        p = int(self.p[v])
        return self.coef[self.coef_off[v]:self.coef_off[v] + 6 * ncoef(p)].reshape(2, 3, ncoef(p))


def _pack(name, ps, coefs, L, centers, **kw) -> Scene:
    ps = np.asarray(ps, dtype=np.int32)
    sizes = np.array([6 * ncoef(int(p)) for p in ps], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    flat = np.concatenate([np.ascontiguousarray(c, dtype=np.float64).ravel() for c in coefs])
    return Scene(name=name, p=ps, coef=flat, coef_off=off, L=np.asarray(L, dtype=np.float64),
                 centers=np.asarray(centers, dtype=np.float64), **kw)


def _vesicle(rng, p, center, R, axes, shape_amp):
    c0 = ellipsoid_coef(p, center, R @ np.diag(axes))
    if shape_amp > 0:
        c0 = c0 + perturbation(rng, p, shape_amp)
    return c0


def _step(rng, p, c0, center, trans, rot_angle, pert_amp):
    R = axis_angle(random_unit(rng), rot_angle) if rot_angle > 0 else np.eye(3)
    c1 = rigid_motion(c0, R, trans, center)
    if pert_amp > 0:
        c1 = c1 + perturbation(rng, p, pert_amp)
    return c1


def two_vesicles(p: int = 8, seed: int = 1, gap: float = 0.05, approach: float = 0.1,
                 pert: float = 0.02, shape_amp: float = 0.01) -> Scene:
    """Two prolate vesicles in free space, surface gap ``gap`` R0 along the
    centre line, closing by ``approach`` R0 over the step (first contact near
    mid-step), plus an SH perturbation of the step."""
    rng = np.random.default_rng(seed)
    a, b = prolate_axes()
    axes = np.array([b, b, a])
    R1, R2 = random_rotation(rng), random_rotation(rng)
    d = random_unit(rng)

    def ray(R, u):  # distance from centre to the ellipsoid surface along u
        A = shape_matrix(R, axes)
        return 1.0 / math.sqrt(float(u @ np.linalg.solve(A, u)))
    c1 = np.zeros(3)
    c2 = d * (ray(R1, d) + ray(R2, -d) + gap * R0_PAPER)
    k1 = _vesicle(rng, p, c1, R1, axes, shape_amp)
    k2 = _vesicle(rng, p, c2, R2, axes, shape_amp)
    k1e = _step(rng, p, k1, c1, np.zeros(3), 0.0, pert)
    k2e = _step(rng, p, k2, c2, -approach * R0_PAPER * d, 0.0, pert)
    coefs = [np.stack([k1, k1e]), np.stack([k2, k2e])]
    return _pack(f"2 vesicles p={p}->{2*p}, gap {gap} R0, approach {approach} R0", [p, p], coefs,
                 np.zeros(3), np.stack([c1, c2]))


def bcc_lattice(nx, ny, nz, a, c):
    """Body-centred lattice of 2 nx ny nz sites in a box (nx a, ny a, nz c)."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    corner = np.stack([ii * a, jj * a, kk * c], -1).reshape(-1, 3)
    centre = corner + np.array([0.5 * a, 0.5 * a, 0.5 * c])
    return np.concatenate([corner, centre]), np.array([nx * a, ny * a, nz * c])


def lattice_scene(name, cells, phi, ps, seed, tilt_deg, trans_amp, rot_deg, pert, shape_amp=0.01,
                  flow_amp=0.0, cubic=True, periodic=True, cell_shape=None) -> Scene:
    """Staggered (body-centred) lattice of prolate vesicles, long axes near z,
    each tilted by a random angle <= tilt_deg (re-drawn until no two
    ellipsoids overlap), in a periodic box at volume fraction phi.  The step is
    a rigid motion: a translation of length trans_amp R0 in a random direction
    plus, if flow_amp > 0, flow_amp times the Taylor-vortex field of Eq. 4.1 at
    the centre; a rotation by <= rot_deg; plus an SH perturbation.  With
    periodic=False the same lattice sits in free space (L = 0)."""
    rng = np.random.default_rng(seed)
    a_ax, b_ax = prolate_axes()
    axes = np.array([b_ax, b_ax, a_ax])
    nx, ny, nz = cells
    n = 2 * nx * ny * nz
    vol = 4.0 / 3.0 * math.pi * a_ax * b_ax * b_ax
    if cell_shape is not None:
        a, c = cell_shape
    elif cubic:   # cube: nx a = nz c
        a = (n * vol / phi) ** (1.0 / 3.0) / nx
        c = nx * a / nz
    else:       # cells stretched like the vesicles, box need not be a cube
        a = (2 * vol / phi / (a_ax / b_ax * 1.05)) ** (1.0 / 3.0)
        c = 2 * vol / phi / (a * a)
    sites, L = bcc_lattice(nx, ny, nz, a, c)
    sites = (sites + rng.uniform(0, 1, 3) * np.array([a, a, c])) % L
    if periodic and np.any(L < 2.0 * (2 * a_ax + 0.5)):
        raise ValueError("periodic box must exceed twice the vesicle extent on every axis")
    rots = [np.eye(3)] * n
    A = [shape_matrix(np.eye(3), axes * 1.02)] * n
    # neighbour lists by minimum image
    nbr = [[] for _ in range(n)]
    reach = 2.2 * a_ax
    for i in range(n):
        d = sites - sites[i]
        if periodic:
            d -= L * np.round(d / L)
        close = np.nonzero(np.linalg.norm(d, axis=1) < reach)[0]
        nbr[i] = [int(j) for j in close if j != i]
    tilt = math.radians(tilt_deg)
    for i in range(n):
        for _ in range(200):
            R = axis_angle(random_unit(rng), rng.uniform(0, tilt)) if tilt > 0 else np.eye(3)
            Ai = shape_matrix(R, axes * 1.02)
            Lp = L if periodic else np.zeros(3)
            if all(not pw_overlap(np.zeros(3), Ai, min_image(sites[j] - sites[i], Lp), A[j]) for j in nbr[i]):
                rots[i], A[i] = R, Ai
                break
    coefs = []
    for i in range(n):
        p = int(ps[i])
        c0 = _vesicle(rng, p, sites[i], rots[i], axes, shape_amp)
        t = trans_amp * R0_PAPER * random_unit(rng)
        if flow_amp > 0:
            x, y, z = 2 * math.pi * sites[i] / L
            t = t + flow_amp * np.array([math.sin(x) * math.cos(y) * math.sin(z),
                                         math.cos(x) * math.sin(y) * math.sin(z), 0.0])
        c1 = _step(rng, p, c0, sites[i], t, math.radians(rng.uniform(0, rot_deg)), pert)
        coefs.append(np.stack([c0, c1]))
    return _pack(name, ps, coefs, L if periodic else np.zeros(3), sites, info=dict(cells=cells, phi=phi, a=a, c=c))


def rsa_scene(name, n, phi, p, seed, trans_amp, rot_deg, pert, shape_amp=0.01) -> Scene:
    """Random sequential addition of randomly oriented prolate vesicles in a
    periodic cube at volume fraction phi (no two ellipsoids, inflated by 2%,
    overlap), each moved by a random rigid motion of trans_amp R0 plus an SH
    perturbation."""
    rng = np.random.default_rng(seed)
    a_ax, b_ax = prolate_axes()
    axes = np.array([b_ax, b_ax, a_ax])
    vol = 4.0 / 3.0 * math.pi * a_ax * b_ax * b_ax
    Lc = (n * vol / phi) ** (1.0 / 3.0)
    L = np.array([Lc, Lc, Lc])
    cs, Rs, As = [], [], []
    tries = 0
    while len(cs) < n:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("RSA did not converge")
        c = rng.uniform(0, Lc, 3)
        R = random_rotation(rng)
        Ai = shape_matrix(R, axes * 1.02)
        ok = True
        for cj, Aj in zip(cs, As):
            d = min_image(cj - c, L)
            if np.linalg.norm(d) > 2.1 * a_ax:
                continue
            if pw_overlap(np.zeros(3), Ai, d, Aj):
                ok = False
                break
        if ok:
            cs.append(c); Rs.append(R); As.append(Ai)
    coefs = []
    for i in range(n):
        c0 = _vesicle(rng, p, cs[i], Rs[i], axes, shape_amp)
        t = trans_amp * R0_PAPER * random_unit(rng)
        c1 = _step(rng, p, c0, cs[i], t, math.radians(rng.uniform(0, 3.0 * rot_deg)), pert)
        coefs.append(np.stack([c0, c1]))
    return _pack(name, [p] * n, coefs, L, np.stack(cs), info=dict(phi=phi, tries=tries))


# --- the named workloads --------------------------------------------------------

def scene_pair(seed: int = 1) -> Scene:
    """2 vesicles, p = 8 -> 16, free space, FP64."""
    return two_vesicles(p=8, seed=seed)


def scene_64(seed: int = 2) -> Scene:
    """64 randomly oriented vesicles at 30% volume fraction, p = 16 -> 32."""
    return rsa_scene("64 vesicles, 30% volume fraction, p=16->32", 64, 0.30, 16, seed,
                     trans_amp=0.05, rot_deg=2.0, pert=0.02)


def scene_1440(seed: int = 3, p: int = 16) -> Scene:
    """1440 vesicles at 58% volume fraction on a staggered 12x12x5 (x2) lattice,
    p = 16 -> 32; the step is tuned for about 2 interfering neighbours per
    vesicle (Sec. 4.3: ~2 contacts per vesicle per step)."""
    n = 1440
    return lattice_scene(f"1440 vesicles, 58% volume fraction, p={p}->{2*p}", (12, 12, 5), 0.58,
                         [p] * n, seed, tilt_deg=3.0, trans_amp=C1440_TRANS, rot_deg=1.0, pert=0.02)


def scene_lattice58(cells=(6, 6, 2), seed: int = 3, p: int = 16) -> Scene:
    """A smaller piece of the 58% lattice workload (same cell shape, density,
    step and order); 2 * prod(cells) vesicles, periodic box."""
    n = 2 * cells[0] * cells[1] * cells[2]
    a = (1440 * 4.0 / 3.0 * math.pi * np.prod(prolate_axes()[0:1]) * prolate_axes()[1] ** 2 / 0.58) ** (1 / 3) / 12
    name = f"{n} vesicles, 58% volume fraction, p={p}->{2*p} (lattice {cells[0]}x{cells[1]}x{cells[2]}x2)"
    return lattice_scene(name, cells, 0.58, [p] * n, seed, tilt_deg=3.0, trans_amp=C1440_TRANS, rot_deg=1.0,
                         pert=0.02, cubic=False, cell_shape=(a, 12 * a / 5))


def scene_4096(seed: int = 4) -> Scene:
    """4096 vesicles at 40% volume fraction, p drawn from {8, 12, 16}, each
    upsampled 2x; Taylor-vortex-shaped step so contacts per vesicle vary."""
    rng = np.random.default_rng(seed + 1000)
    ps = rng.choice(np.array([8, 12, 16]), size=4096)
    return lattice_scene("4096 vesicles, 40% volume fraction, p in {8,12,16}", (16, 16, 8), 0.40, ps, seed,
                         tilt_deg=10.0, trans_amp=C4096_TRANS, rot_deg=2.0, pert=0.02,
                         flow_amp=C4096_FLOW)


def scene_256(seed: int = 5) -> Scene:
    """256 vesicles at 50% volume fraction, p = 12 -> 24 (gradient checks)."""
    return lattice_scene("256 vesicles, 50% volume fraction, p=12->24", (8, 4, 4), 0.50, [12] * 256, seed,
                         tilt_deg=3.0, trans_amp=C256_TRANS, rot_deg=1.0, pert=0.02, cubic=False)


def scene_small(n_side=(2, 1, 1), p: int = 4, seed: int = 7, phi: float = 0.55, trans: float = 0.35,
                periodic: bool = False) -> Scene:
    """Small staggered-lattice cluster for brute-force and parity tests (free
    space unless periodic; a periodic box needs at least 4 x 4 x 2 cells)."""
    nx, ny, nz = n_side
    n = 2 * nx * ny * nz
    return lattice_scene(f"small lattice {n} vesicles p={p}", n_side, phi, [p] * n, seed, tilt_deg=3.0,
                         trans_amp=trans, rot_deg=1.0, pert=0.02, cubic=False, periodic=periodic)


# step sizes (in R0) tuned once so the scenes have the contact density named above
C1440_TRANS = 0.20
C4096_TRANS = 0.30
C4096_FLOW = 2.0
C256_TRANS = 0.40
