"""IPC contact for the oracle (Sec. 7, Eq. barrier), FP64, brute force.

Barrier per primitive pair l (Eq. barrier): B(d) = -(d - dhat)^2 log(d / dhat) for
0 < d < dhat, else 0; the energy adds kappa * sum_l B(d_l) (reading R11: kappa is a
parameter, d the unsquared Euclidean distance). Sec. 7 admits any contact written as an
unconstrained energy, and Table 1 uses an implicit penalty in most scenes; reading R23:
the penalty form replaces B by P(d) = (dhat - d)^2 / 2 for d < dhat (C^1 at dhat, finite at
d = 0), with the same pairs, per-vertex terms and step limit. Pairs (reading R11): surface vertex -
boundary triangle not containing it (VF), boundary edges sharing no vertex (EE), and
vertex - wall plane n.x >= c (VW). Self-contact is included.

Per-vertex terms (reading R12/R19): the barrier enters the vertex gradient exactly
(dB/dx_k = kappa B'(d) dd/dx_k, where by the envelope theorem dd/dx_k = +/- w_k n with the
closest-point weights w_k and unit normal n) and the diagonal block through its
Gauss-Newton part kappa B''(d) (dd/dx_k)(dd/dx_k)^T (B'' > 0 on (0, dhat), so PSD).

Friction (reading R25): the lagged dissipative potential of IPC's friction model on the
vertex-wall pairs. At the start of a step, each surface vertex v near wall p gets a lagged
normal force lam_vp = -kappa E'(d_vp(x_t)) (d < dhat, else 0; E the barrier or penalty), and
D(x) = mu sum_vp lam_vp f0(|P_p (x_v - x_t,v)|), P_p = I - n_p n_p^T the wall's tangent
projector. f0 is C^1: f0(y) = -y^3/(3 eps^2) + y^2/eps + eps/3 for y < eps, y beyond, with
eps = eps_v h (a slip speed eps_v over the step). The walls do not move, so the slip of a
pair is the vertex's own tangential displacement over the step. D enters the energy, the
vertex gradient mu lam f1(y)/y P u (f1 = f0'), and the vertex's diagonal block
mu lam [(f1/y) P + ((f1' y - f1)/y^3) P u u^T P], which is positive semidefinite on both
branches of f0.

Step truncation (reading R11): a surface vertex's step is scaled so that
|delta_v| <= 0.45 min(r_c - dhat, d_min,v), d_min,v = the smallest distance of a pair within
the candidate radius r_c that involves v. No candidate pair's distance can shrink by 90% or
more within one sweep, and no pair outside r_c can come within dhat, so the candidate list
at x^k holds every barrier term along the sweep's line-search segment.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np

# ------------------------------------------------------------------ friction (R25)


def friction_f0(y, eps):
    """C^1 smoothing of |u| below the slip eps: -y^3/(3 eps^2) + y^2/eps + eps/3, y beyond."""
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, -y ** 3 / (3.0 * eps * eps) + y * y / eps + eps / 3.0, y)


def friction_f1(y, eps):
    """f0'(y): -y^2/eps^2 + 2y/eps below eps, 1 beyond."""
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, -y * y / (eps * eps) + 2.0 * y / eps, 1.0)


def friction_f1_over_y(y, eps):
    """f1(y)/y, finite at y = 0 (2/eps)."""
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < eps, -y / (eps * eps) + 2.0 / eps, 1.0 / np.maximum(y, 1e-300))


# ------------------------------------------------------------------ barrier


def barrier(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = (d > 0) & (d < dhat)
    out[m] = -(d[m] - dhat) ** 2 * np.log(d[m] / dhat)
    out[d <= 0] = np.inf
    return out


def barrier_d1(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = (d > 0) & (d < dhat)
    e = d[m] - dhat
    out[m] = -2.0 * e * np.log(d[m] / dhat) - e * e / d[m]
    return out


def barrier_d2(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = (d > 0) & (d < dhat)
    e = d[m] - dhat
    out[m] = -2.0 * np.log(d[m] / dhat) - 4.0 * e / d[m] + e * e / (d[m] * d[m])
    return out


def penalty(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < dhat, 0.5 * (dhat - d) ** 2, 0.0)


def penalty_d1(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < dhat, d - dhat, 0.0)


def penalty_d2(d, dhat):
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < dhat, 1.0, 0.0)


# ------------------------------------------------------------------ closest points


def point_segment(p, a, b):
    """Closest point of segment ab to p: (distance, t) with q = a + t (b - a)."""
    ab = b - a
    L2 = float(ab @ ab)
    t = 0.0 if L2 == 0.0 else float(np.clip((p - a) @ ab / L2, 0.0, 1.0))
    return float(np.linalg.norm(p - (a + t * ab))), t


def point_triangle(p, a, b, c):
    """Closest point of triangle abc to p by its definition: the interior projection if its
    barycentric coordinates are non-negative, else the nearest of the three edges.
    Returns (distance, weights (wa, wb, wc))."""
    n = np.cross(b - a, c - a)
    nn = float(n @ n)
    if nn > 0.0:
        q = p - (p - a) @ n / nn * n
        # barycentric coordinates of q
        v0, v1, v2 = b - a, c - a, q - a
        d00, d01, d11 = v0 @ v0, v0 @ v1, v1 @ v1
        d20, d21 = v2 @ v0, v2 @ v1
        den = d00 * d11 - d01 * d01
        wb = (d11 * d20 - d01 * d21) / den
        wc = (d00 * d21 - d01 * d20) / den
        wa = 1.0 - wb - wc
        if wa >= 0 and wb >= 0 and wc >= 0:
            return float(np.linalg.norm(p - q)), (wa, wb, wc)
    best = None
    for (u, v, iu, iv) in ((a, b, 0, 1), (b, c, 1, 2), (c, a, 2, 0)):
        d, t = point_segment(p, u, v)
        if best is None or d < best[0]:
            w = [0.0, 0.0, 0.0]
            w[iu] = 1.0 - t
            w[iv] = t
            best = (d, tuple(w))
    return best


def segment_segment(p0, p1, q0, q1):
    """Closest points of segments p0p1 and q0q1 by definition: the interior critical point
    of |p(s) - q(t)|^2 if it lies in [0,1]^2, else the best of the four point-segment
    distances on the boundary. Returns (distance, s, t)."""
    d1, d2, r = p1 - p0, q1 - q0, p0 - q0
    a, e, b = d1 @ d1, d2 @ d2, d1 @ d2
    c, f = d1 @ r, d2 @ r
    den = a * e - b * b
    cands = []
    if den > 1e-14 * a * e and a > 0 and e > 0:
        s = (b * f - c * e) / den
        t = (a * f - b * c) / den
        if 0 <= s <= 1 and 0 <= t <= 1:
            cands.append((float(np.linalg.norm(p0 + s * d1 - q0 - t * d2)), float(s), float(t)))
    for s in (0.0, 1.0):
        d, t = point_segment(p0 + s * d1, q0, q1)
        cands.append((d, s, t))
    for t in (0.0, 1.0):
        d, s = point_segment(q0 + t * d2, p0, p1)
        cands.append((d, s, t))
    return min(cands, key=lambda z: z[0])


# ------------------------------------------------------------------ surface and pairs


def surface(tets, X):
    """Boundary faces (used by exactly one tet, oriented outward), their edges, vertices."""
    faces = {}
    for t in np.asarray(tets):
        for k in range(4):
            f = tuple(int(q) for q in np.delete(t, k))
            key = tuple(sorted(f))
            faces.setdefault(key, []).append((f, int(t[k])))
    bf = []
    for key, lst in faces.items():
        if len(lst) != 1:
            continue
        (a, b, c), opp = lst[0]
        n = np.cross(X[b] - X[a], X[c] - X[a])
        if n @ (X[opp] - X[a]) > 0:
            b, c = c, b
        bf.append((a, b, c))
    bf = np.array(sorted(bf, key=lambda f: tuple(sorted(f))), dtype=np.int64).reshape(-1, 3)
    edges = set()
    for a, b, c in bf:
        for u, v in ((a, b), (b, c), (c, a)):
            edges.add((min(u, v), max(u, v)))
    be = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    sv = np.unique(bf.ravel()) if len(bf) else np.zeros(0, np.int64)
    return bf, be, sv


class Contact:
    def __init__(self, tets, X, planes, dhat, kappa, pinned=None, use_penalty=False, friction_mu=0.0,
                 friction_eps_v=1e-3):
        self.faces, self.edges, self.sverts = surface(tets, X)
        self.mu = float(friction_mu)
        self.eps_v = float(friction_eps_v)
        self.fr = None  # lagged friction state (x_t, lam[V, planes], eps) of the current step
        self.planes = np.asarray(planes, dtype=np.float64).reshape(-1, 4)
        self.dhat = float(dhat)
        self.kappa = float(kappa)
        self.pinned = None if pinned is None else np.asarray(pinned).astype(bool)
        # per-pair energy and its d-derivatives: the IPC barrier or the penalty (R23)
        self.e0, self.e1, self.e2 = (penalty, penalty_d1, penalty_d2) if use_penalty else \
            (barrier, barrier_d1, barrier_d2)

    def canonical(self, pairs):
        """Rows (kind, a, b, c, d) in vertex ids: VW (0, v, plane, -1, -1), VF (1, v, face
        vertices ascending), EE (2, edge 1, edge 2; each ascending, edge 1 < edge 2)."""
        rows = []
        for typ, a, b, _ in pairs:
            if typ == 0:
                rows.append((0, a, b, -1, -1))
            elif typ == 1:
                rows.append((1, a, *sorted(int(q) for q in self.faces[b])))
            else:
                e1 = tuple(sorted(int(q) for q in self.edges[a]))
                e2 = tuple(sorted(int(q) for q in self.edges[b]))
                rows.append((2, *min(e1, e2), *max(e1, e2)))
        return sorted(rows)

    def pairs(self, x, radius):
        """Every pair with distance < radius, sorted by (type, a, b): type 0 = VW
        (vertex, plane), 1 = VF (vertex, face index), 2 = EE (edge i < edge j).
        All pairs are enumerated; an axis-aligned box distance (a lower bound of the
        distance) skips the exact closest-point test where it already exceeds the radius."""
        out = []
        sv = self.sverts
        for k, pl in enumerate(self.planes):
            d = x[sv] @ pl[:3] - pl[3]
            for v, dv in zip(sv[d < radius], d[d < radius]):
                out.append((0, int(v), k, float(dv)))
        F, E = self.faces, self.edges
        if len(F):
            flo, fhi = x[F].min(axis=1), x[F].max(axis=1)
            p = x[sv]
            gap = np.maximum(np.maximum(flo[None] - p[:, None], p[:, None] - fhi[None]), 0.0)
            vi, fi = np.nonzero(np.linalg.norm(gap, axis=2) < radius)
            for a, b in zip(vi, fi):
                v = int(sv[a])
                f = F[b]
                if v in f:
                    continue
                d, _ = point_triangle(x[v], x[f[0]], x[f[1]], x[f[2]])
                if d < radius:
                    out.append((1, v, int(b), d))
        if len(E):
            elo, ehi = x[E].min(axis=1), x[E].max(axis=1)
            gap = np.maximum(np.maximum(elo[None] - ehi[:, None], elo[:, None] - ehi[None]), 0.0)
            ii, jj = np.nonzero(np.linalg.norm(gap, axis=2) < radius)
            for i, j in zip(ii, jj):
                if j <= i or len({*E[i], *E[j]}) < 4:
                    continue
                d, _, _ = segment_segment(x[E[i][0]], x[E[i][1]], x[E[j][0]], x[E[j][1]])
                if d < radius:
                    out.append((2, int(i), int(j), d))
        out.sort(key=lambda z: z[:3])
        return out

    def pair_geometry(self, x, pr):
        """(distance, [(vertex, dd/dx_vertex)]) of one pair at positions x."""
        typ, a, b = pr[:3]
        if typ == 0:
            pl = self.planes[b]
            return float(pl[:3] @ x[a] - pl[3]), [(a, pl[:3].copy())]
        if typ == 1:
            f = self.faces[b]
            d, w = point_triangle(x[a], x[f[0]], x[f[1]], x[f[2]])
            q = w[0] * x[f[0]] + w[1] * x[f[1]] + w[2] * x[f[2]]
            n = (x[a] - q) / d if d > 0 else np.zeros(3)
            return d, [(a, n), (f[0], -w[0] * n), (f[1], -w[1] * n), (f[2], -w[2] * n)]
        e1, e2 = self.edges[a], self.edges[b]
        d, s, t = segment_segment(x[e1[0]], x[e1[1]], x[e2[0]], x[e2[1]])
        p = x[e1[0]] + s * (x[e1[1]] - x[e1[0]])
        q = x[e2[0]] + t * (x[e2[1]] - x[e2[0]])
        n = (p - q) / d if d > 0 else np.zeros(3)
        return d, [(e1[0], (1 - s) * n), (e1[1], s * n), (e2[0], -(1 - t) * n), (e2[1], -t * n)]

    def energy(self, x, pairs):
        e = 0.0
        for pr in pairs:
            d, _ = self.pair_geometry(x, pr)
            e += self.kappa * float(self.e0(np.array([d]), self.dhat)[0])
        return e

    def vertex_terms(self, x, pairs, V):
        """Barrier gradient (V,3) and Gauss-Newton diagonal blocks (V,3,3)."""
        g = np.zeros((V, 3))
        H = np.zeros((V, 3, 3))
        for pr in pairs:
            d, J = self.pair_geometry(x, pr)
            if not (0 < d < self.dhat):
                continue
            b1 = self.kappa * float(self.e1(np.array([d]), self.dhat)[0])
            b2 = self.kappa * float(self.e2(np.array([d]), self.dhat)[0])
            for v, jv in J:
                g[v] += b1 * jv
                H[v] += b2 * np.outer(jv, jv)
        return g, H

    def step_limits(self, x, pairs, radius, V):
        """0.45 min(radius - dhat, d_min,v) for surface vertices, inf elsewhere."""
        lim = np.full(V, np.inf)
        lim[self.sverts] = radius - self.dhat
        for pr in pairs:
            d, J = self.pair_geometry(x, pr)
            for v, _ in J:
                lim[v] = min(lim[v], d)
        return 0.45 * lim

    # ---------------------------------------------------------------- friction (R25)

    def lag_friction(self, x_t, h):
        """Lagged normal forces of the step starting at x_t (none when mu = 0)."""
        if self.mu <= 0.0:
            self.fr = None
            return
        V = len(x_t)
        lam = np.zeros((V, len(self.planes)))
        for k, pl in enumerate(self.planes):
            d = x_t[self.sverts] @ pl[:3] - pl[3]
            on = (d > 0) & (d < self.dhat)
            lam[self.sverts[on], k] = -self.kappa * self.e1(d[on], self.dhat)
        if self.pinned is not None:
            lam[self.pinned] = 0.0
        self.fr = (np.array(x_t, dtype=np.float64, copy=True), lam, self.eps_v * h)

    def _slips(self, x):
        x_t, lam, eps = self.fr
        for k, pl in enumerate(self.planes):
            n = pl[:3]
            for v in np.nonzero(lam[:, k] > 0)[0]:
                du = x[v] - x_t[v]
                yield int(v), lam[v, k], du - (du @ n) * n, n, eps

    def friction_energy(self, x):
        if self.fr is None:
            return 0.0
        e = 0.0
        for v, lam, ut, n, eps in self._slips(x):
            e += self.mu * lam * float(friction_f0(np.linalg.norm(ut), eps))
        return e

    def friction_terms(self, x, V):
        """Friction gradient (V,3) and diagonal blocks (V,3,3)."""
        g = np.zeros((V, 3))
        H = np.zeros((V, 3, 3))
        if self.fr is None:
            return g, H
        for v, lam, ut, n, eps in self._slips(x):
            y = float(np.linalg.norm(ut))
            P = np.eye(3) - np.outer(n, n)
            fy = float(friction_f1_over_y(y, eps))
            g[v] += self.mu * lam * fy * ut
            # (f1' y - f1) / y^3: -1/(eps^2 y) below eps, -1/y^2 beyond (no term at y = 0)
            c2 = 0.0 if y == 0.0 else (-1.0 / (eps * eps * y) if y < eps else -1.0 / (y ** 3))
            H[v] += self.mu * lam * (fy * P + c2 * np.outer(ut, ut))
        return g, H

