"""Seeded synthetic inputs: surface meshes, excitation parameters and workload recipes.

This module feeds both the CUDA path and the CPU oracle.  It holds geometry and
bookkeeping only (meshes, pulse parameters, grid placement, random draws) and
none of the method's arithmetic (no basis functions, kernels or matrices).

Workloads follow the benchmark shapes of the paper: PEC spheres meshed with
triangles, a cosine-modulated Gaussian plane wave (Sec. 2.2, Eq. 1) whose band
is f_c +- 3/(2 pi sigma), a delay t_d = 8 sigma (Table I), time step
dt = beta / f_bw with beta = 1/4 (Sec. 3, after Eq. 3) and an auxiliary grid that
encloses the object (Sec. 4).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------


def _orient_outward(v: np.ndarray, f: np.ndarray, center: np.ndarray) -> np.ndarray:
    """Flip faces so that (b-a)x(c-a) points away from ``center`` (convex bodies)."""
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    n = np.cross(b - a, c - a)
    out = np.einsum("ij,ij->i", n, (a + b + c) / 3.0 - center) < 0
    f = f.copy()
    f[out] = f[out][:, [0, 2, 1]]
    return f


def icosphere(sub: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Icosahedron refined ``sub`` times (each triangle split in 4), projected on a sphere.

    Returns ``(V[nv,3] float64, F[nt,3] int32)`` with faces counter-clockwise seen
    from outside.  ``20 * 4**sub`` triangles, ``30 * 4**sub`` edges.
    """
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(x, dtype=np.float64) / math.sqrt(1 + p * p) for x in v]
    faces = list(f)
    for _ in range(sub):
        cache: dict[tuple[int, int], int] = {}

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        faces = nf
    V = np.asarray(verts) * radius + np.asarray(center, dtype=np.float64)
    F = np.asarray(faces, dtype=np.int32)
    F = _orient_outward(V, F, np.asarray(center, dtype=np.float64))
    return V, F.astype(np.int32)


def sphere_array(sub: int, radius: float, pitch: float, nx: int = 4, ny: int = 4):
    """``nx x ny`` spheres in the z=0 plane, centred on the origin, at ``pitch``."""
    Vs, Fs, off = [], [], 0
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * pitch
    for y in ys:
        for x in xs:
            V, F = icosphere(sub, radius, (x, y, 0.0))
            Vs.append(V)
            Fs.append(F + off)
            off += len(V)
    return np.concatenate(Vs), np.concatenate(Fs).astype(np.int32)


def plate_mesh(side: float, n: int):
    """Square plate of side ``side`` in the z = 0 plane, centred on the origin: n x n
    square cells, each split by its (+x, +y) diagonal, faces counter-clockwise about +z.
    The open surface has 3 n^2 - 2 n interior edges (RWG functions): 280, 1160, 4720 and
    19 040 for the 0.1 m cells of the 1, 2, 4 and 8 m plates of Table II."""
    x = (np.arange(n + 1) / n - 0.5) * side
    X, Y = np.meshgrid(x, x, indexing="xy")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros((n + 1) ** 2)], axis=1)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    a = (j * (n + 1) + i).ravel()          # cell corners a (x, y), b (x+1, y), c (x+1, y+1), d (x, y+1)
    b, c, d = a + 1, a + n + 2, a + n + 1
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])
    return V, F.astype(np.int32)


def ellipsoid_mesh(semi_axes=(1.0, 0.5, 0.25), n_points: int = 6668, seed: int = 3,
                   relax_iters: int = 150):
    """Closed ellipsoid surface with nearly uniform point spacing.

    Seeded samples uniform on the unit sphere are mapped onto the ellipsoid and kept
    with probability proportional to the local area scale of that map,
    abc |(u_x/a, u_y/b, u_z/c)| (so the kept points are uniform in ellipsoid area),
    then spread evenly by a repulsion relaxation on the surface (each point pushed away
    from its nearest neighbours and scaled back onto the ellipsoid), triangulated with a
    3-D convex hull and made Delaunay on the surface by edge flips.  Faces are oriented
    outward.  ``E = 3 (V - 2)`` edges, i.e. about ``3 n_points`` RWG unknowns.
    """
    from scipy.spatial import ConvexHull, cKDTree

    ax = np.asarray(semi_axes, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    got = 0
    fmax = ax.prod() * np.linalg.norm(1.0 / ax)
    while got < n_points:
        u = rng.standard_normal((4 * n_points, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        f = ax.prod() * np.linalg.norm(u / ax, axis=1)
        keep = rng.random(len(u)) < f / fmax
        pts.append(u[keep])
        got += int(keep.sum())
    V = np.concatenate(pts)[:n_points] * ax

    def onto(P):
        return P / np.sqrt(((P / ax) ** 2).sum(axis=1, keepdims=True))

    for _ in range(relax_iters):
        d, nb = cKDTree(V).query(V, k=7)
        h = d[:, 1:].mean()
        diff = V[:, None, :] - V[nb[:, 1:]]
        dist = np.maximum(d[:, 1:, None], 1e-12)
        push = (diff / dist ** 3).sum(axis=1)
        step = 0.05 * h ** 3 * push
        V = onto(V + step)
    hull = ConvexHull(V)
    F = _orient_outward(V, hull.simplices.astype(np.int32), np.zeros(3))
    return V, _delaunay_flips(V, F).astype(np.int32)


def _delaunay_flips(V, F, max_pass: int = 100):
    """Lawson edge flips on a closed, consistently oriented triangle surface: an edge
    whose two opposite angles sum to more than pi is replaced by the other diagonal of
    its two triangles, until no such edge is left.  The convex hull of points on an
    ellipsoid is the Delaunay triangulation of the points mapped to the unit sphere
    (hulls are affine invariant), i.e. anisotropic on the ellipsoid itself; the flips
    make it Delaunay in the surface's own angles.  Each pass flips a set of edges that
    share no triangle, largest angle excess first; a flip that would duplicate an
    existing edge is skipped.  Orientation is kept."""
    F = np.array(F, dtype=np.int64)
    nv, nf = len(V), len(F)
    for _ in range(max_pass):
        a = F.reshape(-1)
        b = F[:, [1, 2, 0]].reshape(-1)
        c = F[:, [2, 0, 1]].reshape(-1)
        fi = np.repeat(np.arange(nf), 3)
        key = a * nv + b
        order = np.argsort(key, kind="stable")
        twin = order[np.searchsorted(key[order], b * nv + a)]
        h = np.nonzero(a < b)[0]
        g = twin[h]
        d = c[g]

        def angle_at(p, q, r):  # angle at r of triangle (p, q, r)
            u = V[p] - V[r]
            v = V[q] - V[r]
            cosv = (u * v).sum(1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
            return np.arccos(np.clip(cosv, -1.0, 1.0))

        excess = angle_at(a[h], b[h], c[h]) + angle_at(a[h], b[h], d) - np.pi
        cand = np.nonzero(excess > 1e-12)[0]
        if len(cand) == 0:
            break
        cand = cand[np.argsort(-excess[cand], kind="stable")]
        edges = set((key[a < b]).tolist())
        used = np.zeros(nf, dtype=bool)
        flips = 0
        for j in cand:
            hh, gg = h[j], g[j]
            f1, f2 = fi[hh], fi[gg]
            if used[f1] or used[f2]:
                continue
            ea, eb, ec, ed = int(a[hh]), int(b[hh]), int(c[hh]), int(d[j])
            if ec == ed or min(ec, ed) * nv + max(ec, ed) in edges:
                continue
            F[f1] = (ec, ed, eb)
            F[f2] = (ed, ec, ea)
            used[f1] = used[f2] = True
            edges.discard(min(ea, eb) * nv + max(ea, eb))
            edges.add(min(ec, ed) * nv + max(ec, ed))
            flips += 1
        if flips == 0:
            break
    return F


# ----------------------------------------------------------------------------
# plane-wave draws
# ----------------------------------------------------------------------------


def random_plane_waves(nb: int, seed: int):
    """``nb`` incidence directions uniform on the sphere with a random polarisation.

    k = normalize(N(0, I3)); the polarisation angle psi ~ U[0, 2 pi) is measured in
    the plane orthogonal to k from a fixed reference vector.  PCG64(seed).
    Returns ``(khat[nb,3], phat[nb,3])``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.standard_normal((nb, 3))
    k /= np.linalg.norm(k, axis=1, keepdims=True)
    psi = rng.random(nb) * 2.0 * math.pi
    ref = np.where(np.abs(k[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(k, ref)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(k, e1)
    p = np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2
    return k, p


def seeded_vector(n: int, seed: int) -> np.ndarray:
    """Complex vector with standard normal real and imaginary parts, PCG64(seed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal(n) + 1j * g.standard_normal(n)


def seeded_rows(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct sorted indices below n, PCG64(seed)."""
    return np.sort(np.random.Generator(np.random.PCG64(seed)).choice(n, count, replace=False))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Workload:
    """One benchmark configuration with every derived parameter written out."""

    name: str
    mesh: tuple            # (V, F)
    f_c: float             # carrier (Hz)
    band_frac: float       # band is f_c (1 +- band_frac)
    n_t: int               # time steps
    grid_n: int            # grid nodes per axis
    h: float               # grid spacing (m)
    origin: np.ndarray     # grid node (0,0,0) position
    near_radius: float     # near-zone radius (m) between RWG edge midpoints
    tol: float             # GMRES relative-residual tolerance
    khat: np.ndarray       # [nb,3]
    phat: np.ndarray       # [nb,3]
    order: int = 2         # CPPIF order Q, or the BLIF half-width M
    precision: str = "c64"  # "c128" plain path, "c64" grid path with FP64 outer solve
    beta: float = 0.25
    precond: str = "diag"  # GMRES right preconditioner: "diag" (Sec. 5.1) or "sai"
    precond_radius: float = 0.0  # SAI pattern radius (m); 0: the near radius
    zero_start: bool = False  # GMRES from zero instead of the previous step's currents
    refine: int = 0        # complex64 path: FP64 refinement corrections per step (0: off)
    refine_every: int = 1  # the FP64 residual checked at every k-th step
    autotune: int = 0      # launch shapes: 0 defaults, 1 tuned at setup (cache reused), 2 re-tuned
    rhs_blocked: int = 0   # delayed grid sums by the multilevel blocked schedule (Sec. 4 stage ii)
    eps_r: float = 1.0     # homogeneous background medium (Sec. 2.1); vacuum by default
    mu_r: float = 1.0
    basis: str = "cppif"   # temporal basis: "cppif" (Eq. 3) or "blif" (half-width = order, band = beta)

    @property
    def f_bw(self) -> float:
        return self.band_frac * self.f_c

    @property
    def sigma(self) -> float:
        return 3.0 / (2.0 * math.pi * self.f_bw)

    @property
    def t_d(self) -> float:
        return 8.0 * self.sigma

    @property
    def dt(self) -> float:
        return self.beta / self.f_bw

    @property
    def chi(self) -> float:
        return (self.f_c + self.f_bw) / self.f_bw

    @property
    def nb(self) -> int:
        return int(self.khat.shape[0])


def place_grid(V: np.ndarray, n: int, h: float | None = None):
    """Cubic grid of ``n^3`` nodes centred on the mesh bounding box.

    Without an explicit spacing, ``h = L_max / (n - 5)`` leaves two spare nodes per
    side for a 4-point stencil.  Returns ``(h, origin[3])``.
    """
    lo, hi = V.min(axis=0), V.max(axis=0)
    centre = 0.5 * (lo + hi)
    if h is None:
        h = float((hi - lo).max()) / (n - 5)
    origin = centre - h * (n - 1) / 2.0
    return float(h), origin


def make_workload(name: str, **over) -> Workload:
    """The named benchmark shapes (PEC spheres/ellipsoid/sphere array, CPPIF Q=2; square
    plates, CPPIF Q=3; EFIE throughout)."""
    if name == "sphere480":
        V, F = icosphere(2, 1.0)
        h, o = place_grid(V, 16, 0.15)
        w = dict(mesh=(V, F), f_c=150e6, band_frac=0.5, n_t=200, grid_n=16, h=h, origin=o,
                 near_radius=0.3, tol=1e-6, khat=np.array([[0.0, 0.0, 1.0]]),
                 phat=np.array([[1.0, 0.0, 0.0]]), precision="c128")
    elif name in ("sphere7680", "sphere7680_b64", "sphere7680_wide"):
        V, F = icosphere(4, 1.0)
        h, o = place_grid(V, 64)
        if name == "sphere7680":
            k, p = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
            w = dict(f_c=600e6, band_frac=0.3, n_t=400)
        elif name == "sphere7680_wide":
            # the same sphere and grid at 600 MHz +-60 %: the shorter step gives N_g = 12
            # (a right-hand side with many delays, for the blocked delayed sums)
            k, p = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])
            w = dict(f_c=600e6, band_frac=0.6, n_t=100)
        else:
            k, p = random_plane_waves(64, 0)
            w = dict(f_c=600e6, band_frac=0.1, n_t=300)
        w.update(mesh=(V, F), grid_n=64, h=h, origin=o, near_radius=3 * h, tol=1e-6,
                 khat=k, phat=p, precision="c64")
    elif name == "ellipsoid20k":
        V, F = ellipsoid_mesh()
        h, o = place_grid(V, 96)
        w = dict(mesh=(V, F), f_c=600e6, band_frac=0.3, n_t=500, grid_n=96, h=h, origin=o,
                 near_radius=3 * h, tol=1e-5, khat=np.array([[0.0, 0.0, 1.0]]),
                 phat=np.array([[1.0, 0.0, 0.0]]), precision="c64")
    elif name == "array491k":
        V, F = sphere_array(5, 0.5, 1.5)
        h, o = place_grid(V, 384)
        k, p = random_plane_waves(16, 4)
        w = dict(mesh=(V, F), f_c=1e9, band_frac=0.05, n_t=1000, grid_n=384, h=h, origin=o,
                 near_radius=3 * h, tol=1e-5, khat=k, phat=p, precision="c64")
    elif name.startswith("array_sub"):
        # smaller sphere arrays on the large grid: array_sub<s>_n<N> (4x4 spheres r = 0.5 m)
        s_, n = name[len("array_sub"):].split("_n")
        V, F = sphere_array(int(s_), 0.5, 1.5)
        h, o = place_grid(V, int(n))
        w = dict(mesh=(V, F), f_c=1e9, band_frac=0.05, n_t=50, grid_n=int(n), h=h, origin=o,
                 near_radius=3 * h, tol=1e-5, khat=np.array([[0.0, 0.0, 1.0]]),
                 phat=np.array([[1.0, 0.0, 0.0]]), precision="c64")
    elif name.startswith("plate"):
        # square PEC plates of Table II (0.1 m cells, 3 n^2 - 2 n RWG), EFIE (alpha = 1,
        # Sec. 5.1), the chi ~ 20 pulse of Table I (f_c = 285 MHz, sigma = 1/(10 pi) us,
        # so f_c + 3/(2 pi sigma) = 300 MHz) and CPPIF Q = 3 (Table III), at normal incidence
        side, grid = {"plate280": (1.0, 16), "plate1160": (2.0, 32), "plate4720": (4.0, 64),
                      "plate19k": (8.0, 96), "plate306k": (32.0, 384)}[name]
        V, F = plate_mesh(side, int(round(side / 0.1)))
        h, o = place_grid(V, grid)
        f_bw = 3.0 / (2.0 * math.pi * (1e-6 / (10.0 * math.pi)))
        w = dict(mesh=(V, F), f_c=285e6, band_frac=f_bw / 285e6, n_t=80, grid_n=grid, h=h, origin=o,
                 near_radius=3 * h, tol=1e-6, khat=np.array([[0.0, 0.0, -1.0]]),
                 phat=np.array([[1.0, 0.0, 0.0]]), order=3, precision="c64")
    elif name.startswith("sphere_sub"):
        # small parity cases: sphere_sub<s>_n<N>  (radius 1 m, 600 MHz +-30 %)
        s, n = name[len("sphere_sub"):].split("_n")
        V, F = icosphere(int(s), 1.0)
        h, o = place_grid(V, int(n))
        w = dict(mesh=(V, F), f_c=over.pop("f_c", 300e6), band_frac=0.3, n_t=60, grid_n=int(n),
                 h=h, origin=o, near_radius=3 * h, tol=1e-6,
                 khat=np.array([[0.0, 0.0, 1.0]]), phat=np.array([[1.0, 0.0, 0.0]]),
                 precision="c64")
    else:
        raise KeyError(name)
    w.update(over)
    return Workload(name=name, **w)
