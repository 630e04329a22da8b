"""Star-shaped islands on the unit sphere, drawn from a seeded generator.

Each island k is a cap bounded by the curve

    x(t) = cos r(t) c_k + sin r(t) (cos t e1 + sin t e2),   r(t) = r0 (1 + a cos(kf t)),

in geodesic polar coordinates about its centre c_k, with the frame
e1 = normalise(z x c) (x-hat instead of z-hat when |c_z| > 0.9) and e2 = c x e1,
so the curve runs counter-clockwise about c_k seen from outside the sphere.
Nodes are equispaced in t (the parameter alpha of Sec. 5).  The first and
second t-derivatives are analytic.

Island family (the same for every workload): r0 ~ U[0.05, 0.25] s(M),
a ~ U[0, 0.3], kf ~ U{2..8}, with s(M) = min(1, sqrt(16/M)) so that the islands
cover about 10% of the sphere whatever M is (at s = 1, M = 16 the expected cap
area is about 0.082 per island).  Centres are uniform on the sphere and kept
only if their angle to every accepted centre is at least 1.2 (R_i + R_j) with
R = r0 (1 + a).

By default every point is rotated so that the centre of island 0 sits at the
north pole (Sec. 3 assumes without loss of generality that the first curve
encircles the pole); the frame, sources and targets are built before that
rotation so the data do not depend on the pole choice.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Geometry:
    M: int
    island_ptr: np.ndarray  # int64 (M+1), CSR offsets of the islands' nodes
    x: np.ndarray  # (N, 3) nodes on the sphere
    dx: np.ndarray  # (N, 3) dx/dt
    d2x: np.ndarray  # (N, 3) d2x/dt2
    centres: np.ndarray  # (M, 3) geodesic-polar centres, inside each island
    r0: np.ndarray
    amp: np.ndarray
    kfreq: np.ndarray
    e1: np.ndarray  # (M, 3) frames (after rotation)
    e2: np.ndarray
    rotation: np.ndarray = field(default_factory=lambda: np.eye(3))
    # "star": r(t) = r0 (1 + amp cos(kfreq t)); "ellipse": semi-axes (axes[:, 0], axes[:, 1])
    # with the major axis at angle axes[:, 2] from e1
    shape: str = "star"
    axes: np.ndarray | None = None

    def radius(self, k: int, t):
        """The island's geodesic radius r(t) about its centre."""
        if self.shape == "ellipse":
            a, b, ph = self.axes[k]
            u = np.asarray(t) - ph
            return a * b / np.sqrt((b * np.cos(u)) ** 2 + (a * np.sin(u)) ** 2)
        return self.r0[k] * (1.0 + self.amp[k] * np.cos(self.kfreq[k] * np.asarray(t)))

    def rmax(self, k: int) -> float:
        if self.shape == "ellipse":
            return float(max(self.axes[k, 0], self.axes[k, 1]))
        return float(self.r0[k] * (1.0 + self.amp[k]))

    def rmin(self, k: int) -> float:
        if self.shape == "ellipse":
            return float(min(self.axes[k, 0], self.axes[k, 1]))
        return float(self.r0[k] * (1.0 - self.amp[k]))

    @property
    def N(self) -> int:
        return int(self.island_ptr[-1])

    @property
    def nodes_per_island(self) -> np.ndarray:
        return np.diff(self.island_ptr)

    def island_of_node(self) -> np.ndarray:
        return np.repeat(np.arange(self.M), self.nodes_per_island)


def _frame(c: np.ndarray):
    ref = np.array([0.0, 0.0, 1.0]) if abs(c[2]) <= 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(ref, c)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(c, e1)
    return e1, e2


def rotation_to_pole(c: np.ndarray) -> np.ndarray:
    """Rotation matrix R with R c = (0, 0, 1) (Rodrigues' formula)."""
    c = np.asarray(c, dtype=np.float64)
    c = c / np.linalg.norm(c)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(c, z)
    s = np.linalg.norm(v)
    cth = float(c @ z)
    if s < 1e-15:
        if cth > 0:
            return np.eye(3)
        return np.diag([1.0, -1.0, -1.0])  # half turn about x
    kx = v / s
    Kx = np.array([[0, -kx[2], kx[1]], [kx[2], 0, -kx[0]], [-kx[1], kx[0], 0]])
    return np.eye(3) + s * Kx + (1.0 - cth) * (Kx @ Kx)


def apply_rotation(R: np.ndarray, pts: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(pts, dtype=np.float64) @ R.T)


def _curve(c, e1, e2, r0, a, kf, n):
    t = TWO_PI * np.arange(n) / n
    r = r0 * (1.0 + a * np.cos(kf * t))
    rp = -r0 * a * kf * np.sin(kf * t)
    rpp = -r0 * a * kf * kf * np.cos(kf * t)
    ct, st = np.cos(t)[:, None], np.sin(t)[:, None]
    u = ct * e1 + st * e2
    v = -st * e1 + ct * e2
    cr, sr = np.cos(r)[:, None], np.sin(r)[:, None]
    rp_, rpp_ = rp[:, None], rpp[:, None]
    C = c[None, :]
    x = cr * C + sr * u
    dx = -rp_ * sr * C + rp_ * cr * u + sr * v
    d2x = (-rpp_ * sr - rp_ ** 2 * cr) * C + (rpp_ * cr - rp_ ** 2 * sr - sr) * u + 2.0 * rp_ * cr * v
    return x, dx, d2x


def _draw_centres(rng, R, max_draws=1_000_000):
    M = len(R)
    cs = np.zeros((M, 3))
    draws = 0
    for i in range(M):
        while True:
            draws += 1
            if draws > max_draws:
                raise RuntimeError(f"could not place {M} islands without overlap")
            c = rng.normal(size=3)
            c /= np.linalg.norm(c)
            if i == 0:
                break
            ang = np.arccos(np.clip(cs[:i] @ c, -1.0, 1.0))
            if np.all(ang >= 1.2 * (R[:i] + R[i])):
                break
        cs[i] = c
    return cs


def star_caps(seed: int, M: int, nodes, *, r0=None, amp=None, kfreq=None,
              r0_range=(0.05, 0.25), amp_range=(0.0, 0.3), k_range=(2, 8),
              scale=None, pole: str | None = "first") -> Geometry:
    """Draw M star caps with the given nodes per island (int or array of M ints).

    r0, amp, kfreq may be given explicitly (arrays of length M); otherwise they
    are drawn per island in the order (r0, a, kf) before any centre is drawn.
    """
    rng = np.random.default_rng(seed)
    if scale is None:
        scale = min(1.0, float(np.sqrt(16.0 / M)))
    if r0 is None:
        r0 = np.empty(M)
        amp = np.empty(M)
        kfreq = np.empty(M, dtype=np.int64)
        for i in range(M):
            r0[i] = rng.uniform(*r0_range) * scale
            amp[i] = rng.uniform(*amp_range)
            kfreq[i] = rng.integers(k_range[0], k_range[1] + 1)
    r0 = np.asarray(r0, dtype=np.float64)
    amp = np.asarray(amp, dtype=np.float64)
    kfreq = np.asarray(kfreq, dtype=np.int64)
    R = r0 * (1.0 + amp)
    centres = _draw_centres(rng, R)
    nodes = np.broadcast_to(np.asarray(nodes, dtype=np.int64), (M,)).copy()
    ptr = np.zeros(M + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(nodes)
    N = int(ptr[-1])
    x = np.empty((N, 3))
    dx = np.empty((N, 3))
    d2x = np.empty((N, 3))
    E1 = np.empty((M, 3))
    E2 = np.empty((M, 3))
    for i in range(M):
        e1, e2 = _frame(centres[i])
        E1[i], E2[i] = e1, e2
        a, b = ptr[i], ptr[i + 1]
        x[a:b], dx[a:b], d2x[a:b] = _curve(centres[i], e1, e2, r0[i], amp[i], kfreq[i], int(nodes[i]))
    g = Geometry(M=M, island_ptr=ptr, x=x, dx=dx, d2x=d2x, centres=centres.copy(),
                 r0=r0, amp=amp, kfreq=kfreq, e1=E1, e2=E2)
    if pole == "first":
        g = rotated(g, rotation_to_pole(centres[0]))
    elif pole is not None:
        raise ValueError(pole)
    return g


def rotated(g: Geometry, R: np.ndarray) -> Geometry:
    """The same islands with every point and frame vector multiplied by R."""
    return Geometry(M=g.M, island_ptr=g.island_ptr.copy(), x=apply_rotation(R, g.x),
                    dx=apply_rotation(R, g.dx), d2x=apply_rotation(R, g.d2x),
                    centres=apply_rotation(R, g.centres), r0=g.r0.copy(), amp=g.amp.copy(),
                    kfreq=g.kfreq.copy(), e1=apply_rotation(R, g.e1), e2=apply_rotation(R, g.e2),
                    rotation=R @ g.rotation, shape=g.shape,
                    axes=None if g.axes is None else g.axes.copy())


def _point_at(g: Geometry, k: int, rho: float, t: float) -> np.ndarray:
    c, e1, e2 = g.centres[k], g.e1[k], g.e2[k]
    return np.cos(rho) * c + np.sin(rho) * (np.cos(t) * e1 + np.sin(t) * e2)


def pair_sources(g: Geometry, k_plus: int = 0, k_minus: int | None = None, frac: float = 0.5):
    """A +1 / -1 pair of point sources strictly inside islands.

    For a single island (k_minus is None or equal to k_plus) the +1 source is
    the island centre and the -1 source lies at geodesic distance frac * r_min
    from it along e1.  Otherwise each source lies at frac * r_min from its
    island's centre along that island's e1.
    """
    if k_minus is None or k_minus == k_plus:
        k = k_plus
        rmin = g.rmin(k)
        p = g.centres[k].copy()
        q = _point_at(g, k, frac * rmin, 0.0)
        return np.stack([p, q]), np.array([1.0, -1.0]), np.array([k, k])
    pts = []
    for k in (k_plus, k_minus):
        rmin = g.rmin(k)
        pts.append(_point_at(g, k, frac * rmin, 0.0))
    return np.stack(pts), np.array([1.0, -1.0]), np.array([k_plus, k_minus])


def random_pair_sources(g: Geometry, rng: np.random.Generator):
    """A +1 / -1 pair in two random islands (both in island 0 when M = 1),
    each at a random geodesic radius below 0.8 r_min and a random angle."""
    if g.M == 1:
        ks = (0, 0)
    else:
        ks = tuple(int(v) for v in rng.choice(g.M, size=2, replace=False))
    pts = []
    for k in ks:
        rmin = g.rmin(k)
        pts.append(_point_at(g, k, rng.uniform(0.1, 0.8) * rmin, rng.uniform(0, TWO_PI)))
    return np.stack(pts), np.array([1.0, -1.0]), np.array(ks)


def _inside_island(g: Geometry, y: np.ndarray) -> np.ndarray:
    """Exact test in geodesic polar coordinates about each centre: inside iff rho < r(t)."""
    inside = np.zeros(len(y), dtype=bool)
    for k in range(g.M):
        c, e1, e2 = g.centres[k], g.e1[k], g.e2[k]
        rho = np.arccos(np.clip(y @ c, -1.0, 1.0))
        near = rho < g.rmax(k) + 1e-12
        if not near.any():
            continue
        t = np.arctan2(y[near] @ e2, y[near] @ e1)
        r = g.radius(k, t)
        inside[np.flatnonzero(near)[rho[near] < r]] = True
    return inside


def targets_off_islands(g: Geometry, T: int, seed: int, clearance: float = 5.0) -> np.ndarray:
    """T uniform points on the sphere outside every island and at chord distance
    at least clearance * h_k |x'_j| from every node j of every island k."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    h = np.repeat(TWO_PI / g.nodes_per_island, g.nodes_per_island)
    guard = clearance * h * np.linalg.norm(g.dx, axis=1)
    tree = cKDTree(g.x)
    gmax = float(guard.max())
    out = []
    while len(out) < T:
        y = rng.normal(size=(4 * T, 3))
        y /= np.linalg.norm(y, axis=1)[:, None]
        y = y[~_inside_island(g, y)]
        for pt in y:
            idx = tree.query_ball_point(pt, gmax)
            if idx:
                d = np.linalg.norm(g.x[idx] - pt, axis=1)
                if np.any(d < guard[idx]):
                    continue
            out.append(pt)
            if len(out) == T:
                break
    return np.ascontiguousarray(np.array(out))


def _ellipse_curve(c, e1, e2, a, b, ph, n):
    """The curve of geodesic radius r(t) = a b / sqrt(b^2 cos^2 u + a^2 sin^2 u), u = t - ph
    (an ellipse with semi-axes a, b in geodesic polar coordinates), with its analytic
    t-derivatives."""
    t = TWO_PI * np.arange(n) / n
    u = t - ph
    D = (b * np.cos(u)) ** 2 + (a * np.sin(u)) ** 2
    D1 = (a * a - b * b) * np.sin(2.0 * u)
    D2 = 2.0 * (a * a - b * b) * np.cos(2.0 * u)
    r = a * b * D ** -0.5
    rp = -0.5 * a * b * D ** -1.5 * D1
    rpp = a * b * (0.75 * D ** -2.5 * D1 ** 2 - 0.5 * D ** -1.5 * D2)
    ct, st = np.cos(t)[:, None], np.sin(t)[:, None]
    uu = ct * e1 + st * e2
    vv = -st * e1 + ct * e2
    cr, sr = np.cos(r)[:, None], np.sin(r)[:, None]
    rp_, rpp_ = rp[:, None], rpp[:, None]
    C = c[None, :]
    x = cr * C + sr * uu
    dx = -rp_ * sr * C + rp_ * cr * uu + sr * vv
    d2x = (-rpp_ * sr - rp_ ** 2 * cr) * C + (rpp_ * cr - rp_ ** 2 * sr - sr) * uu + 2.0 * rp_ * cr * vv
    return x, dx, d2x


def fibonacci_centres(M: int) -> np.ndarray:
    """M points spread regularly over the sphere (a Fibonacci lattice)."""
    i = np.arange(M) + 0.5
    z = 1.0 - 2.0 * i / M
    phi = np.pi * (3.0 - np.sqrt(5.0)) * np.arange(M)
    rxy = np.sqrt(np.clip(1.0 - z * z, 0.0, None))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def ellipse_islands(seed: int, M: int, nodes, *, pole: str | None = "first") -> Geometry:
    """M elliptical islands spread regularly over the sphere with random semi-axes and
    orientations (the shape of the paper's first and third examples, whose exact axes are
    not given): centres on a Fibonacci lattice, semi-axes a, b ~ U[0.15, 0.38] d and
    orientation ~ U[0, pi), d the lattice's smallest angular spacing, so that every pair
    keeps the star-cap family's clearance (angle >= 1.2 (R_i + R_j))."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    centres = fibonacci_centres(M)
    if M > 1:
        dd, _ = cKDTree(centres).query(centres, k=2)
        d = 2.0 * np.arcsin(np.clip(dd[:, 1].min() / 2.0, 0.0, 1.0))
    else:
        d = 1.0
    axes = np.empty((M, 3))
    for k in range(M):
        axes[k, 0] = rng.uniform(0.15, 0.38) * d
        axes[k, 1] = rng.uniform(0.15, 0.38) * d
        axes[k, 2] = rng.uniform(0.0, np.pi)
    nodes = np.broadcast_to(np.asarray(nodes, dtype=np.int64), (M,)).copy()
    ptr = np.zeros(M + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(nodes)
    N = int(ptr[-1])
    x, dx, d2x = np.empty((N, 3)), np.empty((N, 3)), np.empty((N, 3))
    E1, E2 = np.empty((M, 3)), np.empty((M, 3))
    for k in range(M):
        e1, e2 = _frame(centres[k])
        E1[k], E2[k] = e1, e2
        a_, b_ = ptr[k], ptr[k + 1]
        x[a_:b_], dx[a_:b_], d2x[a_:b_] = _ellipse_curve(centres[k], e1, e2, *axes[k], int(nodes[k]))
    rmax = axes[:, :2].max(axis=1)
    g = Geometry(M=M, island_ptr=ptr, x=x, dx=dx, d2x=d2x, centres=centres.copy(),
                 r0=rmax, amp=np.zeros(M), kfreq=np.zeros(M, dtype=np.int64), e1=E1, e2=E2,
                 shape="ellipse", axes=axes)
    if pole == "first":
        g = rotated(g, rotation_to_pole(centres[0]))
    elif pole is not None:
        raise ValueError(pole)
    return g


def random_density(N: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(N)


# --- the five workload families -------------------------------------------------

def config_geometry(name: str, **kw) -> Geometry:
    """Geometry of a named workload.

    C1: one cap r = 0.4 (1 + 0.2 cos 5t), random centre, N = 256 (seed 1).
    C2: 16 caps of the family, 512 nodes each, N = 8192 (seed 2).
    C3: 2^e caps x 1024 nodes (e = 10..14, default 10) (seed 3); kw 'M'.
    C5: 256 caps x 512 nodes, N = 131072 (seed 5).
    """
    if name == "C1":
        n = kw.get("nodes", 256)
        return star_caps(1, 1, n, r0=[0.4], amp=[0.2], kfreq=[5], pole=kw.get("pole", "first"))
    if name == "C2":
        return star_caps(2, kw.get("M", 16), kw.get("nodes", 512), pole=kw.get("pole", "first"))
    if name == "C3":
        return star_caps(3, kw.get("M", 1024), kw.get("nodes", 1024), pole=kw.get("pole", "first"))
    if name == "C5":
        return star_caps(5, kw.get("M", 256), kw.get("nodes", 512), pole=kw.get("pole", "first"))
    raise KeyError(name)


def batch_instances(seed: int = 4, count: int = 512, nrhs: int = 16, max_islands: int = 64,
                    nodes_range=(64, 1024)):
    """Independent geometries of uneven size with several source pairs each: per
    instance M ~ U{1..max_islands}, nodes per island round(exp U(ln a, ln b)) for
    nodes_range = (a, b), and nrhs +1/-1 source pairs in random islands (both in
    island 0 when M = 1).  Returns a list of (Geometry, [(points, strengths), ...])."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = np.log(nodes_range[0]), np.log(nodes_range[1])
    for _ in range(count):
        M = int(rng.integers(1, max_islands + 1))
        nodes = np.rint(np.exp(rng.uniform(lo, hi, size=M))).astype(np.int64)
        g = star_caps(int(rng.integers(0, 2**31 - 1)), M, nodes)
        srng = np.random.default_rng(int(rng.integers(0, 2**31 - 1)))
        pairs = []
        for _ in range(nrhs):
            p, gam, _ = random_pair_sources(g, srng)
            pairs.append((p, gam))
        out.append((g, pairs))
    return out
