"""Seeded synthetic scene generators shared by the CUDA path's tests/bench and the oracle.

This module only builds inputs: lattice coordinates, tetrahedral connectivity, per-tet
material parameters, pinned masks and initial velocities. It holds none of the method's
arithmetic (no masses, no rest-shape inverses, no energies); each side derives those itself.

The workloads mirror the paper's experiments (Sec. 8, Table 1): voxelised tetrahedral
solids split into Kuhn tetrahedra, dropped under gravity, with a soft/stiff material mix.
Every random draw uses numpy's PCG64 generator keyed by an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# The six Kuhn tetrahedra of a unit cube: each walks from corner 000 to corner 111 along
# one permutation of the axes. Corner code = x + 2y + 4z.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _kuhn_local():
    tets = []
    for p in _PERMS:
        c = [0, 0, 0]
        path = [0]
        for ax in p:
            c[ax] = 1
            path.append(c[0] + 2 * c[1] + 4 * c[2])
        # orientation: even permutations give positive volume with this walk
        a, b, d = np.eye(3)[p[0]], np.eye(3)[p[0]] + np.eye(3)[p[1]], np.ones(3)
        if np.linalg.det(np.stack([a, b, d], axis=1)) < 0:
            path[1], path[2] = path[2], path[1]
        tets.append(path)
    return np.array(tets, dtype=np.int64)


KUHN = _kuhn_local()


@dataclass
class Scene:
    """A tetrahedral scene. Arrays are in the caller's (generator's) vertex order."""
    name: str
    X: np.ndarray            # (V,3) float64 rest positions, also the initial positions
    tets: np.ndarray         # (T,4) int32
    youngs: np.ndarray       # (T,) float64 Pa
    poisson: np.ndarray      # (T,) float64
    density: np.ndarray      # (T,) float64 kg/m^3
    pinned: np.ndarray       # (V,) uint8
    v0: np.ndarray           # (V,3) float64 initial velocity
    dt: float = 1.0 / 120.0
    gravity: tuple = (0.0, 0.0, -9.8)
    planes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # (n, c): n.x >= c
    dhat: float = 1e-3
    kappa: float = 1e5
    contact: int = 0
    x0: np.ndarray | None = None  # initial positions if different from X

    @property
    def n_vertices(self):
        return int(self.X.shape[0])

    @property
    def n_tets(self):
        return int(self.tets.shape[0])


def voxel_mesh(mask: np.ndarray, cell: tuple, origin=(0.0, 0.0, 0.0)):
    """Kuhn-split every filled cell of a boolean (nx,ny,nz) cell mask.

    Returns rest positions (V,3) and tets (T,4); vertices are numbered by first use in
    x-fastest lattice order, cells are visited in the same order.
    """
    mask = np.asarray(mask, dtype=bool)
    nx, ny, nz = mask.shape
    cx, cy, cz = np.nonzero(mask.transpose(2, 1, 0))  # z, y, x order -> x fastest
    cz, cy, cx = cx, cy, cz
    order = np.lexsort((cx, cy, cz))
    cx, cy, cz = cx[order], cy[order], cz[order]
    corner = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)])
    lat = np.stack([cx, cy, cz], axis=1)[:, None, :] + corner[None, :, :]  # (C,8,3)
    key = (lat[..., 2] * (ny + 1) + lat[..., 1]) * (nx + 1) + lat[..., 0]
    uniq, inv = np.unique(key.ravel(), return_inverse=True)
    inv = inv.reshape(key.shape)
    tets = inv[:, KUHN].reshape(-1, 4)
    gx = uniq % (nx + 1)
    gy = (uniq // (nx + 1)) % (ny + 1)
    gz = uniq // ((nx + 1) * (ny + 1))
    X = np.stack([gx * cell[0], gy * cell[1], gz * cell[2]], axis=1) + np.asarray(origin)
    return X.astype(np.float64), tets.astype(np.int32)


def kuhn_grid(nvx, nvy, nvz, size):
    """A box of nvx*nvy*nvz lattice vertices spanning `size`, every cell Kuhn-split."""
    cell = (size[0] / (nvx - 1), size[1] / (nvy - 1), size[2] / (nvz - 1))
    return voxel_mesh(np.ones((nvx - 1, nvy - 1, nvz - 1), bool), cell)


def voxel_sphere(radius, cells_across, center=(0.0, 0.0, 0.0)):
    """Cells of a cube lattice whose centres lie inside the sphere, Kuhn-split."""
    n = int(cells_across)
    h = 2.0 * radius / n
    c = (np.arange(n) + 0.5) * h - radius
    gx, gy, gz = np.meshgrid(c, c, c, indexing="ij")
    mask = gx ** 2 + gy ** 2 + gz ** 2 <= radius ** 2
    origin = np.asarray(center, dtype=np.float64) - radius
    return voxel_mesh(mask, (h, h, h), origin)


def _uniform_material(T, E, nu, rho):
    return (np.full(T, float(E)), np.full(T, float(nu)), np.full(T, float(rho)))


def cube_scene():
    """5x5x5-vertex cube of side 0.1 m, 384 Kuhn tets, top face pinned, at rest."""
    X, tets = kuhn_grid(5, 5, 5, (0.1, 0.1, 0.1))
    E, nu, rho = _uniform_material(len(tets), 1e5, 0.4, 1000.0)
    pinned = (np.abs(X[:, 2] - X[:, 2].max()) < 1e-12).astype(np.uint8)
    return Scene("cube", X, tets, E, nu, rho, pinned, np.zeros_like(X))


def beam_scene(nvx=100, nvy=20, nvz=20, length=0.1, width=0.02, E=1e7, nu=0.45,
               vel_sigma=0.05, seed=0):
    """Clamped stiff beam: long axis x, the x=0 face clamped, random initial velocity."""
    X, tets = kuhn_grid(nvx, nvy, nvz, (length, width, width))
    Ev, nuv, rho = _uniform_material(len(tets), E, nu, 1000.0)
    pinned = (X[:, 0] < 1e-12).astype(np.uint8)
    rng = np.random.default_rng(seed)
    v0 = rng.normal(0.0, vel_sigma, size=X.shape)
    v0[pinned.astype(bool)] = 0.0
    return Scene("beam", X, tets, Ev, nuv, rho, pinned, v0)


def box_planes(size=(1.0, 1.0, 2.0)):
    """Floor and four side walls of an open-top box, as (normal, offset): n.x >= c."""
    return np.array([
        [0, 0, 1, 0.0],
        [1, 0, 0, 0.0], [-1, 0, 0, -size[0]],
        [0, 1, 0, 0.0], [0, -1, 0, -size[1]],
    ], dtype=np.float64)


def sphere_centres(n_spheres=10, radius=0.1, seed=0, dhat=1e-3):
    """Seeded centres of the spheres scene: uniform in [0.15,0.85]^2 x [0.5,1.9], rejected
    until every pair is at least 2 radius + 2 dhat apart."""
    rng = np.random.default_rng(seed)
    centres = []
    while len(centres) < n_spheres:
        c = rng.uniform([0.15, 0.15, 0.5], [0.85, 0.85, 1.9])
        if all(np.linalg.norm(c - d) >= 2 * radius + 2 * dhat for d in centres):
            centres.append(c)
    return centres


def sphere_of_scene(k, n_spheres=10, radius=0.1, cells_across=48, seed=0, dhat=1e-3,
                    E_stiff=2e6, E_soft=1e5):
    """Sphere k of spheres_scene alone (same coordinates and material, no contact): the
    spheres are separate bodies, so a body-by-body computation can take them one at a time."""
    Xs, ts = voxel_sphere(radius, cells_across)
    c = sphere_centres(n_spheres, radius, seed, dhat)[k]
    T = len(ts)
    E = E_stiff if k < n_spheres // 2 else E_soft
    return Scene(f"sphere{k}", Xs + c, ts.astype(np.int32), np.full(T, E), np.full(T, 0.4),
                 np.full(T, 1000.0), np.zeros(len(Xs), np.uint8), np.zeros_like(Xs))


def spheres_scene(n_spheres=10, radius=0.1, cells_across=48, seed=0, dhat=1e-3,
                  E_stiff=2e6, E_soft=1e5, contact=1):
    """Ten voxel spheres at seeded separated positions above a 1x1x2 m box.

    Spheres 0..n/2-1 are stiff, the rest soft; all share one lattice shape.
    """
    Xs, ts = voxel_sphere(radius, cells_across)
    centres = sphere_centres(n_spheres, radius, seed, dhat)
    Xl, tl, El = [], [], []
    for k, c in enumerate(centres):
        Xl.append(Xs + c)
        tl.append(ts + k * len(Xs))
        El.append(np.full(len(ts), E_stiff if k < n_spheres // 2 else E_soft))
    X = np.concatenate(Xl)
    tets = np.concatenate(tl).astype(np.int32)
    E = np.concatenate(El)
    T = len(tets)
    return Scene("spheres", X, tets, E, np.full(T, 0.4), np.full(T, 1000.0),
                 np.zeros(len(X), np.uint8), np.zeros_like(X), planes=box_planes(),
                 dhat=dhat, contact=contact)


def _blob_params(index, t_min, t_max):
    rng = np.random.default_rng(index)
    k = int(rng.integers(1, 7))
    centres = rng.uniform(0.0, 0.1, size=(k, 3))
    radii = rng.uniform(0.02, 0.05, size=k)
    target = float(np.exp(rng.uniform(np.log(t_min), np.log(t_max))))
    E = float(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
    nu = float(rng.uniform(0.3, 0.48))
    return k, centres, radii, target, E, nu


def blob_tet_target(index, t_min=1e3, t_max=5e4):
    """The tet count blob_scene(index) aims at (its mesh is within 10% of it), without
    building the mesh: enough to balance scenes across ranks."""
    return _blob_params(index, t_min, t_max)[3]


def blob_scene(index, t_min=1e3, t_max=5e4):
    """One seeded random voxel blob (union of 1-6 spheres), bottom layer pinned.

    The tet count is drawn log-uniform in [t_min, t_max]; the cell size is bisected
    until the blob's tet count is within 10% of that target.
    """
    k, centres, radii, target, E, nu = _blob_params(index, t_min, t_max)
    lo = (centres - radii[:, None]).min(0)
    hi = (centres + radii[:, None]).max(0)

    def build(cell):
        n = np.maximum(np.ceil((hi - lo) / cell).astype(int), 1)
        cc = [lo[d] + (np.arange(n[d]) + 0.5) * cell for d in range(3)]
        gx, gy, gz = np.meshgrid(*cc, indexing="ij")
        P = np.stack([gx, gy, gz], -1)
        mask = np.zeros(gx.shape, bool)
        for c, r in zip(centres, radii):
            mask |= ((P - c) ** 2).sum(-1) <= r * r
        return mask

    a, b = 1e-3, 5e-2
    mask = build(b)
    for _ in range(40):
        cell = np.sqrt(a * b)
        mask = build(cell)
        t = 6 * int(mask.sum())
        if abs(t - target) <= 0.1 * target:
            break
        if t > target:
            a = cell
        else:
            b = cell
    X, tets = voxel_mesh(mask, (cell, cell, cell), lo)
    T = len(tets)
    pinned = (np.abs(X[:, 2] - X[:, 2].min()) < 1e-9 * max(1.0, abs(X[:, 2].min()))).astype(np.uint8)
    return Scene(f"blob{index}", X, tets, np.full(T, E), np.full(T, nu), np.full(T, 1000.0),
                 pinned, np.zeros_like(X))


def small_beam_scene(nvx=9, nvy=3, nvz=3, E=1e6, nu=0.45, seed=0, vel_sigma=0.05):
    """A few-hundred-DOF clamped beam for fast tests (same recipe as the stiff beam)."""
    return beam_scene(nvx, nvy, nvz, 0.1, 0.02, E, nu, vel_sigma, seed)


def random_cubature(X, tets, pinned, n_cub=4, seed=0, w_max=2.0, u_sigma=0.3):
    """Seeded synthetic cubature records for sweep-parity inputs (not a precompute).

    For every free vertex: n_cub distinct elements drawn from its own body that do not
    touch it, weights uniform in [0, w_max), and U_bar blocks with entries N(0, u_sigma^2)
    (zero rows at pinned corners). Element draws are restricted to a random pool of at most
    256 elements per body, as the library's pools are.
    """
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    V = len(X)
    T = len(tets)
    rows = np.repeat(tets[:, :1], 3, axis=1).ravel()
    cols = tets[:, 1:].ravel()
    G = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(V, V))
    nb, body = csg.connected_components(G, directed=False)
    tbody = body[tets[:, 0]]
    rng = np.random.default_rng(seed)
    pools = {}
    for b in range(nb):
        el = np.nonzero(tbody == b)[0]
        pools[b] = np.sort(rng.choice(el, size=min(256, len(el)), replace=False))
    pin = np.asarray(pinned).astype(bool)
    free = np.nonzero(~pin)[0]
    elem = -np.ones((V, n_cub), np.int64)
    n_draw = 4 * n_cub
    cand = np.empty((len(free), n_draw), np.int64)
    for b in range(nb):
        sel = body[free] == b
        cand[sel] = pools[b][rng.integers(0, len(pools[b]), size=(int(sel.sum()), n_draw))]
    ok = ~np.any(tets[cand] == free[:, None, None], axis=2)
    for j in range(n_draw):  # first n_cub distinct, non-incident draws per vertex
        c = cand[:, j]
        dup = np.any(elem[free] == c[:, None], axis=1)
        slot = (elem[free] >= 0).sum(axis=1)
        take = ok[:, j] & ~dup & (slot < n_cub)
        elem[free[take], slot[take]] = c[take]
    used = elem >= 0
    weight = np.where(used, rng.uniform(0.0, w_max, size=(V, n_cub)), 0.0)
    ubar = rng.normal(0.0, u_sigma, size=(V, n_cub, 4, 3, 3))
    ubar[~used] = 0.0
    corner_pinned = used[..., None] & pin[tets[np.maximum(elem, 0)]]
    ubar[corner_pinned] = 0.0
    return elem, weight, ubar


def perturbed_state(X, pinned, scale, seed=0):
    """x^k = X + smooth-ish random displacement of the free vertices (parity inputs)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(0.0, scale, size=X.shape)
    d[np.asarray(pinned).astype(bool)] = 0.0
    return X + d


def drop_scene(nv=4, size=0.02, gap=5e-4, speed=0.3, E=1e5, dhat=1e-3, kappa=1e4):
    """A small free block just above the floor, moving down: exercises the wall barrier."""
    X, tets = kuhn_grid(nv, nv, nv, (size, size, size))
    X = X + np.array([0.3, 0.3, gap])
    T = len(tets)
    v0 = np.zeros_like(X)
    v0[:, 2] = -speed
    return Scene("drop", X, tets, np.full(T, E), np.full(T, 0.4), np.full(T, 1000.0),
                 np.zeros(len(X), np.uint8), v0, planes=box_planes(), dhat=dhat, kappa=kappa, contact=1)


def slide_scene(nv=3, size=0.02, gap=9.8e-4, speed=0.5, E=1e5, dhat=1e-3, kappa=1e4):
    """A small free block resting within dhat of the floor (the gap puts the barrier force
    near its weight), sliding along it: exercises wall friction."""
    X, tets = kuhn_grid(nv, nv, nv, (size, size, size))
    X = X + np.array([0.3, 0.3, gap])
    T = len(tets)
    v0 = np.zeros_like(X)
    v0[:, 0] = speed
    v0[:, 1] = 0.4 * speed
    return Scene("slide", X, tets, np.full(T, E), np.full(T, 0.4), np.full(T, 1000.0),
                 np.zeros(len(X), np.uint8), v0, planes=box_planes(), dhat=dhat, kappa=kappa, contact=1)


def stack_scene(nv=3, size=0.02, gap=1.5e-3, speed=0.3, E=1e5, dhat=1e-3, kappa=1e4):
    """Two small blocks, the upper one moving down onto the lower one resting on the floor
    (vertex-face and edge-edge pairs between bodies, and the floor)."""
    X, tets = kuhn_grid(nv, nv, nv, (size, size, size))
    off = np.array([0.003, 0.002, 0.0])
    Xa = np.vstack([X + [0.3, 0.3, 0.8 * dhat], X + [0.3, 0.3, size + gap] + off])
    ta = np.vstack([tets, tets + len(X)]).astype(np.int32)
    T = len(ta)
    v0 = np.zeros_like(Xa)
    v0[len(X):, 2] = -speed
    return Scene("stack", Xa, ta, np.full(T, E), np.full(T, 0.4), np.full(T, 1000.0),
                 np.zeros(len(Xa), np.uint8), v0, planes=box_planes(), dhat=dhat, kappa=kappa, contact=1)


@dataclass
class ClothScene:
    """A triangle-mesh cloth. Arrays are in the generator's vertex order."""
    name: str
    X: np.ndarray            # (V,3) float64 rest positions, also the initial positions
    tris: np.ndarray         # (F,3) int32
    youngs: float            # Pa
    poisson: float
    thickness: float         # m
    density: float           # kg/m^3
    bend: float              # bending stiffness (N m)
    pinned: np.ndarray       # (V,) uint8
    v0: np.ndarray           # (V,3)
    dt: float = 1.0 / 120.0
    gravity: tuple = (0.0, 0.0, -9.8)
    planes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # walls n.x >= c
    dhat: float = 1e-3
    kappa: float = 1e5


def cloth_grid(n, size):
    """n x n vertices on a flat square of side `size` in the z = 0 plane, every cell split
    into two triangles along alternating diagonals."""
    g = np.linspace(0.0, size, n)
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    X = np.hstack([X, np.zeros((len(X), 1))])
    tris = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return X, np.array(tris, dtype=np.int32)


def cloth_scene(n=21, size=0.5, youngs=1e6, thickness=5e-4, bend=1e-5, seed=0, vel_sigma=0.0):
    """A square cloth held at two adjacent corners, released flat under gravity."""
    X, tris = cloth_grid(n, size)
    pinned = np.zeros(len(X), np.uint8)
    pinned[0] = pinned[(n - 1) * n] = 1
    v0 = np.random.default_rng(seed).normal(0.0, vel_sigma, X.shape) if vel_sigma > 0 else np.zeros_like(X)
    v0[pinned.astype(bool)] = 0.0
    return ClothScene("cloth", X, tris, youngs, 0.3, thickness, 200.0, bend, pinned, v0)


def cloth_floor_scene(n=11, size=0.2, gap=6e-4, youngs=1e5, kappa=1e2):
    """A small free cloth lying flat just above the floor (z >= 0, within dhat), under gravity:
    exercises the cloth's wall barrier."""
    X, tris = cloth_grid(n, size)
    X = X + np.array([0.3, 0.3, gap])
    return ClothScene("cloth_floor", X, tris, youngs, 0.3, 5e-4, 200.0, 1e-5, np.zeros(len(X), np.uint8),
                      np.zeros_like(X), planes=np.array([[0.0, 0.0, 1.0, 0.0]]), dhat=1e-3, kappa=kappa)

