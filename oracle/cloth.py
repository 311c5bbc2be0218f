"""Cloth for the oracle: StVK membrane triangles and a quadratic bending energy (the cloth
material the paper's Table 1 caption lists for its cloth example), stepped by the per-vertex
Jacobi sweep with the global line search (readings R17, R26). FP64, plain numpy.

Reading R26 (the paper names the materials but gives no formulas):
- Membrane (Saint Venant-Kirchhoff, plane stress). Per triangle with rest corners X_0..2, an
  orthonormal frame (t1, t2) of its plane gives the 2x2 rest edge matrix D_m (columns: the
  edges X_1 - X_0, X_2 - X_0 in that frame) and area A. F = [x_1 - x_0, x_2 - x_0] D_m^-1
  (3x2) = sum_a x_a b_a^T, with b_1, b_2 the rows of D_m^-1 and b_0 = -(b_1 + b_2).
  E = (F^T F - I)/2, Psi = mu tr(E^2) + lam/2 tr(E)^2 with membrane moduli
  mu = Y t / (2 (1 + nu)), lam = Y t nu / (1 - nu^2) (Young's modulus Y, thickness t);
  energy A Psi. Gradient at corner a: A F S b_a with S = 2 mu E + lam tr(E) I. Diagonal
  block: A [(b_a^T S b_a) I + (mu + lam) (F b_a)(F b_a)^T + mu |b_a|^2 F F^T].
- Bending (quadratic, isometric): for each interior edge (x_0, x_1) with opposite vertices
  x_2 (first triangle) and x_3 (second), rest cotangent weights
  K = (cot a_1 + cot c_1, cot a_0 + cot c_0, -(cot a_0 + cot a_1), -(cot c_0 + cot c_1)),
  a_j the rest angle at x_j in triangle (x_0, x_1, x_2), c_j the one in (x_0, x_1, x_3);
  energy k_b 3/(A_0 + A_1) |sum_i K_i x_i|^2 / 2. K sums to zero and, for a flat rest
  hinge, annihilates its rest positions, so every affine image of a flat rest sheet has
  zero bending energy. The energy is quadratic in x: gradient k K_i w, diagonal block
  k K_i^2 I (w = sum K_j x_j).
- Mass: rho t A / 3 per corner. Implicit Euler as for the solids (Sec. 3).
- Sweep: per free vertex, D_v = -H_vv^-1 g_v with H_vv = m_v/h^2 I + the positive
  semidefinite part of the summed membrane blocks + the bending blocks (StVK's blocks can
  be indefinite under compression); then the global Armijo search of R17 along D (no
  cubature correction: the Ubar records of Eq. u are built on tets only).
- Walls (optional): every free vertex against every wall plane n.x >= c with the IPC
  barrier of Sec. 7 (kappa B(d), d = n.x - c, as for the solids, reading R11): gradient
  kappa B'(d) n, Gauss-Newton block kappa B''(d) n n^T, and the same step limit
  |D_v| <= 0.45 min(r_c - dhat, d_min,v), r_c = 2 dhat, d_min,v the smallest wall distance
  below r_c. The line search evaluates the barrier exactly per trial.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .contact import barrier, barrier_d1, barrier_d2
from .fem import psd_clamp

LS_TRIALS = 8
ARMIJO_C = 1e-4


class Cloth:
    def __init__(self, X, tris, youngs, poisson, thickness, density, bend, pinned=None, planes=None, dhat=1e-3,
                 kappa=1e5):
        self.planes = np.zeros((0, 4)) if planes is None else np.asarray(planes, dtype=np.float64).reshape(-1, 4)
        self.dhat, self.kappa, self.rc = float(dhat), float(kappa), 2.0 * float(dhat)
        X = np.asarray(X, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.X, self.tris = X, tris
        Fn = len(tris)
        self.youngs = np.broadcast_to(np.asarray(youngs, dtype=np.float64), (Fn,)).copy()
        nu = np.broadcast_to(np.asarray(poisson, dtype=np.float64), (Fn,))
        th = np.broadcast_to(np.asarray(thickness, dtype=np.float64), (Fn,))
        rho = np.broadcast_to(np.asarray(density, dtype=np.float64), (Fn,))
        self.mu = self.youngs * th / (2.0 * (1.0 + nu))
        self.lam = self.youngs * th * nu / (1.0 - nu * nu)
        e1 = X[tris[:, 1]] - X[tris[:, 0]]
        e2 = X[tris[:, 2]] - X[tris[:, 0]]
        n = np.cross(e1, e2)
        self.area = 0.5 * np.linalg.norm(n, axis=1)
        t1 = e1 / np.linalg.norm(e1, axis=1)[:, None]
        t2 = np.cross(n / np.linalg.norm(n, axis=1)[:, None], t1)
        Dm = np.stack([np.stack([np.sum(e1 * t1, 1), np.sum(e2 * t1, 1)], 1),
                       np.stack([np.sum(e1 * t2, 1), np.sum(e2 * t2, 1)], 1)], 1)  # [F][2][2]
        Di = np.linalg.inv(Dm)
        # b_a (a = 0..2) as rows: F = sum_a x_a b_a^T
        self.b = np.stack([-(Di[:, 0] + Di[:, 1]), Di[:, 0], Di[:, 1]], 1)  # [F][3][2]
        V = len(X)
        self.mass = np.zeros(V)
        np.add.at(self.mass, tris.ravel(), np.repeat(rho * th * self.area / 3.0, 3))
        self.pinned = np.zeros(V, bool) if pinned is None else np.asarray(pinned).astype(bool)
        self.free = np.nonzero(~self.pinned)[0]
        self.hinges, self.K, self.kb = self._hinges(float(np.mean(np.atleast_1d(bend))))

    def _hinges(self, bend):
        """Interior edges (x_0, x_1, x_2, x_3), their cotangent weights and stiffnesses."""
        X, tris = self.X, self.tris
        opp = {}
        for f, t in enumerate(tris):
            for k in range(3):
                a, b = int(t[k]), int(t[(k + 1) % 3])
                opp.setdefault((min(a, b), max(a, b)), []).append((int(t[(k + 2) % 3]), f))
        H, K, kb = [], [], []

        def cot(p, q, r):  # cotangent of the angle at p in triangle (p, q, r)
            u, v = q - p, r - p
            return float(u @ v) / float(np.linalg.norm(np.cross(u, v)))

        for (a, b), lst in sorted(opp.items()):
            if len(lst) != 2:
                continue
            (c, f0), (d, f1) = lst
            x0, x1, x2, x3 = X[a], X[b], X[c], X[d]
            ca0, ca1 = cot(x0, x1, x2), cot(x1, x0, x2)
            cc0, cc1 = cot(x0, x1, x3), cot(x1, x0, x3)
            H.append((a, b, c, d))
            K.append((ca1 + cc1, ca0 + cc0, -(ca0 + ca1), -(cc0 + cc1)))
            kb.append(3.0 * bend / (self.area[f0] + self.area[f1]))
        return (np.array(H, dtype=np.int64).reshape(-1, 4), np.array(K).reshape(-1, 4), np.array(kb))

    @property
    def V(self):
        return self.X.shape[0]

    def deformation(self, x):
        return np.einsum("fai,faj->fij", x[self.tris], self.b)  # [F][3][2]

    def membrane(self, x):
        """Per-triangle energy, F, Green strain E and S = 2 mu E + lam tr(E) I."""
        F = self.deformation(x)
        E = 0.5 * (np.einsum("fki,fkj->fij", F, F) - np.eye(2)[None])
        tr = E[:, 0, 0] + E[:, 1, 1]
        psi = self.mu * np.einsum("fij,fij->f", E, E) + 0.5 * self.lam * tr * tr
        S = 2.0 * self.mu[:, None, None] * E + (self.lam * tr)[:, None, None] * np.eye(2)[None]
        return self.area * psi, F, E, S

    def bending_w(self, x):
        return np.einsum("hi,hik->hk", self.K, x[self.hinges])  # [H][3]

    def wall_distances(self, x):
        """[free vertices][planes] distances n.x - c."""
        return x[self.free] @ self.planes[:, :3].T - self.planes[:, 3][None, :]

    def energy(self, x, z, h):
        em, _, _, _ = self.membrane(x)
        w = self.bending_w(x)
        d = (x - z)[self.free]
        e = float(np.sum(em) + 0.5 * np.sum(self.kb * np.sum(w * w, 1)) +
                  np.sum(0.5 * self.mass[self.free] / h ** 2 * np.sum(d * d, 1)))
        if len(self.planes):
            e += self.kappa * float(np.sum(barrier(self.wall_distances(x), self.dhat)))
        return e

    def gradient(self, x, z, h):
        _, F, _, S = self.membrane(x)
        P = np.einsum("fij,fjk->fik", F, S)  # F S [F][3][2]
        ge = self.area[:, None, None] * np.einsum("fik,fak->fai", P, self.b)
        g = np.zeros_like(x)
        np.add.at(g, self.tris.ravel(), ge.reshape(-1, 3))
        w = self.bending_w(x)
        gb = (self.kb[:, None, None] * self.K[:, :, None]) * w[:, None, :]
        np.add.at(g, self.hinges.ravel(), gb.reshape(-1, 3))
        g += self.mass[:, None] / h ** 2 * (x - z)
        if len(self.planes):
            b1 = self.kappa * barrier_d1(self.wall_distances(x), self.dhat)  # [free][planes]
            g[self.free] += b1 @ self.planes[:, :3]
        g[self.pinned] = 0.0
        return g

    def diag_blocks(self, x, h, project=True):
        """H_vv: inertia, membrane blocks (summed, then their PSD part), bending blocks."""
        _, F, _, S = self.membrane(x)
        Fb = np.einsum("fij,faj->fai", F, self.b)  # F b_a [F][3][3]
        bSb = np.einsum("faj,fjk,fak->fa", self.b, S, self.b)
        bb = np.einsum("faj,faj->fa", self.b, self.b)
        FFt = np.einsum("fij,fkj->fik", F, F)
        lm = (self.mu + self.lam)[:, None, None, None]
        Hm = self.area[:, None, None, None] * (bSb[:, :, None, None] * np.eye(3)[None, None] +
                                               lm * np.einsum("fai,faj->faij", Fb, Fb) +
                                               (self.mu[:, None] * bb)[:, :, None, None] * FFt[:, None])
        Hd = np.zeros((self.V, 3, 3))
        np.add.at(Hd, self.tris.ravel(), Hm.reshape(-1, 3, 3))
        if project:
            Hd = psd_clamp(Hd)
        kb = (self.kb[:, None] * self.K ** 2).ravel()
        np.add.at(Hd, self.hinges.ravel(), kb[:, None, None] * np.eye(3)[None])
        Hd += (self.mass / h ** 2)[:, None, None] * np.eye(3)[None]
        if len(self.planes):
            b2 = self.kappa * barrier_d2(self.wall_distances(x), self.dhat)
            n = self.planes[:, :3]
            Hd[self.free] += np.einsum("vp,pi,pj->vij", b2, n, n)
        return Hd

    def step_limits(self, x):
        """0.45 min(r_c - dhat, d_min) per free vertex (inf without walls), reading R11."""
        lim = np.full(self.V, np.inf)
        if len(self.planes):
            d = self.wall_distances(x)
            dm = np.where(d < self.rc, d, np.inf).min(axis=1)
            lim[self.free] = 0.45 * np.minimum(self.rc - self.dhat, dm)
        return lim


def inertia_target(x_t, v_t, h, gravity):
    return x_t + h * v_t + h * h * np.asarray(gravity, dtype=np.float64)[None, :]


def direction(c: Cloth, x, z, h):
    g = c.gradient(x, z, h)
    H = c.diag_blocks(x, h)
    D = np.zeros_like(x)
    lim = c.step_limits(x)
    for v in c.free:
        D[v] = -np.linalg.solve(H[v], g[v])
        n = np.linalg.norm(D[v])
        if n > lim[v]:
            D[v] *= lim[v] / n
    return D, g


def line_search(c: Cloth, x, z, h, D, g):
    """Global Armijo backtracking on E along D (reading R17), a_j = 2^-j, j < 8; no move if
    every trial fails."""
    e0 = c.energy(x, z, h)
    slope = float(np.sum(g * D))
    for j in range(LS_TRIALS):
        a = 1.0 / (1 << j)
        if c.energy(x + a * D, z, h) - e0 <= ARMIJO_C * a * slope:
            return a * D
    return np.zeros_like(D)


def run_sweeps(c: Cloth, x, z, h, n=1, line_search_on=True):
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(n):
        D, g = direction(c, x, z, h)
        x = x + (line_search(c, x, z, h, D, g) if line_search_on else D)
    return x


@dataclass
class StepResult:
    x: np.ndarray
    v: np.ndarray
    sweeps: int
    residuals: list = field(default_factory=list)
    converged: bool = False


def step(c: Cloth, x_t, v_t, h, gravity, rel_tol=1e-4, max_sweeps=100):
    """One implicit-Euler step from x^0 = x_t: sweeps until |g(x^k)| <= rel_tol |g(x^0)| or
    max_sweeps (the same stopping rule as the solids' step)."""
    z = inertia_target(x_t, v_t, h, gravity)
    x = np.array(x_t, dtype=np.float64, copy=True)
    res, g0, k, conv = [], None, 0, False
    while True:
        D, g = direction(c, x, z, h)
        gn = float(np.linalg.norm(g[c.free]))
        g0 = gn if g0 is None else g0
        r = gn / g0 if g0 > 0 else 0.0
        res.append(r)
        if r <= rel_tol or g0 == 0.0:
            conv = True
            break
        if k >= max_sweeps:
            break
        x = x + line_search(c, x, z, h, D, g)
        k += 1
    return StepResult(x, (x - x_t) / h, k, res, conv)
