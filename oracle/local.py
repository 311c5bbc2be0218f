"""Per-vertex evaluation of the JGS2 direction for very large meshes (Secs. 4-5, 8.1).

Same definitions as sweep.direction, evaluated for a few sampled vertices using only
the tets around them, so that full-size meshes (millions of tets) can be checked vertex
by vertex. Plain loops over the handful of tets involved; FP64.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np

from . import fem, sweep


class LocalMesh:
    def __init__(self, X, tets, youngs, poisson, density, pinned):
        self.X = np.asarray(X, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.E = np.asarray(youngs, dtype=np.float64)
        self.nu = np.asarray(poisson, dtype=np.float64)
        self.rho = np.asarray(density, dtype=np.float64)
        self.pinned = np.asarray(pinned).astype(bool)
        order = np.argsort(self.tets.ravel(), kind="stable")
        self._inc_tet = order // 4
        self._inc_start = np.searchsorted(self.tets.ravel()[order], np.arange(self.X.shape[0] + 1))

    def incident(self, v):
        return self._inc_tet[self._inc_start[v]:self._inc_start[v + 1]]

    def rest(self, t):
        """(b (4,3), V_e, mu, lam') of tet t."""
        tv = self.tets[t]
        Dm = np.stack([self.X[tv[k]] - self.X[tv[0]] for k in (1, 2, 3)], axis=1)
        B = np.linalg.inv(Dm)
        b = np.vstack([-B.sum(axis=0), B])
        mu, lp = fem.lame(self.E[t], self.nu[t])
        return b, np.linalg.det(Dm) / 6.0, float(mu), float(lp)

    def mass(self, v):
        return sum(self.rho[t] * self.rest(t)[1] / 4.0 for t in self.incident(v))

    def F(self, t, x):
        b, _, _, _ = self.rest(t)
        return np.einsum("ai,aj->ij", x[self.tets[t]], b)

    def vertex_terms(self, v, x, z, h):
        """g_v, H_vv (exact diagonal block), F_v (volume-weighted mean) at x."""
        g = np.zeros(3)
        H = np.zeros((3, 3))
        Fs = np.zeros((3, 3))
        W = 0.0
        m = 0.0
        for t in self.incident(v):
            b, vol, mu, lp = self.rest(t)
            F = np.einsum("ai,aj->ij", x[self.tets[t]], b)
            c = int(np.nonzero(self.tets[t] == v)[0][0])
            P = fem.snh_P(F, mu, lp)
            A = fem.snh_dPdF(F, mu, lp).reshape(3, 3, 3, 3)
            g += vol * P @ b[c]
            H += vol * np.einsum("j,ijkl,l->ik", b[c], A, b[c])
            Fs += vol * F
            W += vol
            m += self.rho[t] * vol / 4.0
        g += m / h ** 2 * (x[v] - z[v])
        H += m / h ** 2 * np.eye(3)
        if self.pinned[v]:
            g[:] = 0.0
        return g, H, Fs / W

    def element_hessian(self, t, x, h):
        b, vol, mu, lp = self.rest(t)
        F = np.einsum("ai,aj->ij", x[self.tets[t]], b)
        A = fem.snh_dPdF(F, mu, lp).reshape(3, 3, 3, 3)
        He = vol * np.einsum("aj,ijkl,cl->aick", b, A, b).reshape(12, 12)
        return He + self.rho[t] * vol / 4.0 / h ** 2 * np.eye(12)

    def direction(self, i, x, z, h, elem, weight, ubar):
        """(D_i, D_J,i) of the JGS2 sweep at vertex i for its cubature records."""
        g, H, Fi = self.vertex_terms(i, x, z, h)
        DJ = np.linalg.solve(H, -g)
        Ri = sweep.polar_rotation(Fi)
        Ht = np.zeros((3, 3))
        gt = np.zeros(3)
        for s in range(len(elem)):
            e = int(elem[s])
            if e < 0:
                continue
            Us = []
            ga = []
            for a_loc, a in enumerate(self.tets[e]):
                ga_, _, Fa = self.vertex_terms(a, x, z, h)
                Ra = sweep.polar_rotation(Fa)
                Us.append(Ra @ ubar[s, a_loc] @ Ri.T)
                ga.append(ga_ if not self.pinned[a] else np.zeros(3))
            U = np.vstack(Us)
            Ht += weight[s] * U.T @ self.element_hessian(e, x, h) @ U
            gt += weight[s] * U.T @ np.concatenate(ga)
        try:
            np.linalg.cholesky(H + Ht)
            D = np.linalg.solve(H + Ht, -(g + gt))
        except np.linalg.LinAlgError:
            D = DJ
        return D, DJ
