"""Offline stage: rest Hessian, full-coordinate subspace U_bar, cubature training (Secs. 4-6).

* H_bar: Hessian of E at the rest shape over free DOFs, inertia M/h^2 included (reading
  R2: without it a free-floating body's H_bar is singular). Block-diagonal per body.
* U_bar_i = -H_bar^{-1} S_i^T G_i with G_i = -(S_i H_bar^{-1} S_i^T)^{-1}       (Eq. u, Sec. 6)
  i.e. Y_i = H_bar^{-1} S_i^T, A_i = S_i Y_i, U_bar_i = Y_i A_i^{-1}. Rows at pinned
  vertices are zero (pinned vertices are not DOFs).
* Training poses: the n_train lowest eigenvectors q_t of H_bar (Sec. 5, last paragraph).
* Cubature (Eq. cubature_weight, Sec. 5), reading R3 "asm": for pose t the sampled element
  e contributes c_e^(t) = sum_{a in e} U_bar_{i,a}^T (H_bar q_t)_a and the target is the
  complement sum b^(t) = sum_{a != i} U_bar_{i,a}^T (H_bar q_t)_a, which has the closed form
  A_i^{-1} q_{t,i} - lambda_t q_{t,i} (because H_bar U_bar_i = S_i^T A_i^{-1}). Rows of pose
  t are divided by |b^(t)|; weights come from non-negative least squares (library NNLS).
* Greedy selection (Sec. 5): each round draws n_cand candidates from the body's element
  pool (elements not incident to i and not yet selected, reading R4), keeps the one with
  the lowest NNLS residual (ties: lowest element id), and stops at n_cub elements or when
  the relative residual drops below nnls_tol (1%, Sec. 5).
  Reading R6b: the candidates of every vertex of a body come from one seeded pool of
  n_pool elements of that body (n_pool >= body size recovers a draw from all elements).
  Draws are keyed by body-local indices (the rank of a vertex / element among its body's
  vertices / elements in caller order), so identical bodies get identical records:
  pool = draw(keyed(seed, 2^32-1, 0), local elements, n_pool), candidates of local vertex l
  in round r = draw(keyed(seed, l, r), eligible pool elements in ascending order, n_cand).

Dense linear algebra (numpy) for the small meshes the tests use.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.optimize

from . import fem, rng


@dataclass
class Cubature:
    """Per-vertex cubature records in caller vertex order (pinned vertices: elem = -1)."""
    elem: np.ndarray      # (V, n_cub) int64, -1 = unused slot
    weight: np.ndarray    # (V, n_cub) float64
    ubar: np.ndarray      # (V, n_cub, 4, 3, 3) float64: U_bar_{i,a} for the element's corners
    residual: np.ndarray  # (V,) relative NNLS residual of the final set (nan for pinned)

    @property
    def n_cub(self):
        return self.elem.shape[1]


def rest_hessian(mesh: fem.Mesh, h):
    """H_bar = grad^2 E(X) on free DOFs (reading R2: includes M/h^2)."""
    return fem.global_hessian(mesh, mesh.X, h, psd=False, dense=True)


def ubar_all(mesh: fem.Mesh, Hbar):
    """Full-coordinate precompute (Eq. u): for every free vertex i, Y_i = H^-1 S_i^T,
    A_i = S_i Y_i and U_bar_i = Y_i A_i^{-1}. Returns (Ubar (nf, N, 3), A (nf, 3, 3))."""
    N = Hbar.shape[0]
    Hinv = np.linalg.inv(Hbar)
    nf = N // 3
    Ub = np.empty((nf, N, 3))
    A = np.empty((nf, 3, 3))
    for d in range(nf):
        Y = Hinv[:, 3 * d:3 * d + 3]
        Ai = Y[3 * d:3 * d + 3]
        A[d] = Ai
        Ub[d] = Y @ np.linalg.inv(Ai)
    return Ub, A


def body_eigs(mesh: fem.Mesh, Hbar, body, n_train):
    """Lowest n_train eigenpairs of H_bar restricted to one body's free DOFs."""
    vid = mesh.free[mesh.body_of_vertex[mesh.free] == body]
    dofs = (3 * mesh.dof_of[vid][:, None] + np.arange(3)[None, :]).ravel()
    Hb = Hbar[np.ix_(dofs, dofs)]
    lam, Q = np.linalg.eigh(Hb)
    k = min(n_train, len(lam))
    q = np.zeros((k, Hbar.shape[0]))
    q[:, dofs] = Q[:, :k].T
    return lam[:k], q


def body_pool(mesh: fem.Mesh, body, n_pool, seed):
    """Seeded pool of a body's elements (body-local draw keyed (2^32-1, 0)), ascending ids."""
    elems = np.nonzero(mesh.body_of_tet == body)[0]
    g = rng.keyed(seed, 0xFFFFFFFF, 0)
    local = rng.draw_without_replacement(g, list(range(len(elems))), n_pool)
    return sorted(int(elems[j]) for j in local)


def fit_system(mesh: fem.Mesh, i, Ub_i, A_i, lam, q, cand_elems):
    """Rows of Eq. cubature_weight for vertex i: columns c_e^(t)/|b^(t)|, target b^(t)/|b^(t)|."""
    d = mesh.dof_of[i]
    qi = q[:, 3 * d:3 * d + 3]                             # (T,3)
    b = qi @ np.linalg.inv(A_i).T - lam[:, None] * qi      # A_i^-1 q_ti - lam_t q_ti
    nb = np.linalg.norm(b, axis=1)
    keep = nb > 1e-12 * max(nb.max(), 1e-300)
    cols = []
    for e in cand_elems:
        c = np.zeros_like(b)
        for a in mesh.tets[e]:
            da = mesh.dof_of[a]
            if da < 0:
                continue
            Uia = Ub_i[3 * da:3 * da + 3]                   # (3,3) rows of vertex a
            c += lam[:, None] * (q[:, 3 * da:3 * da + 3] @ Uia)   # U^T (H q)_a = lam U^T q_a
        cols.append((c[keep] / nb[keep, None]).ravel())
    y = (b[keep] / nb[keep, None]).ravel()
    return np.array(cols).T if cols else np.zeros((y.size, 0)), y


def train_cubature(mesh: fem.Mesh, h, n_cub=4, n_train=20, n_cand=32, n_pool=256,
                   nnls_tol=0.01, seed=0, Hbar=None):
    """Greedy NNLS cubature (Sec. 5) for every free vertex; returns a Cubature record set."""
    if Hbar is None:
        Hbar = rest_hessian(mesh, h)
    Ub, A = ubar_all(mesh, Hbar)
    V = mesh.V
    elem = -np.ones((V, n_cub), dtype=np.int64)
    weight = np.zeros((V, n_cub))
    ubar = np.zeros((V, n_cub, 4, 3, 3))
    resid = np.full(V, np.nan)
    eig = {b: body_eigs(mesh, Hbar, b, n_train) for b in range(mesh.n_bodies)}
    pools = {b: body_pool(mesh, b, n_pool, seed) for b in range(mesh.n_bodies)}
    incident = [set() for _ in range(V)]
    for e, t in enumerate(mesh.tets):
        for a in t:
            incident[a].add(e)
    local_index = np.zeros(V, dtype=np.int64)
    for b in range(mesh.n_bodies):
        vb = np.nonzero(mesh.body_of_vertex == b)[0]
        local_index[vb] = np.arange(len(vb))
    for i in mesh.free:
        d = mesh.dof_of[i]
        body = mesh.body_of_vertex[i]
        lam, q = eig[body]
        sel, w, res = [], np.zeros(0), 1.0
        for r in range(n_cub):
            if res < nnls_tol:
                break
            eligible = [e for e in pools[body] if e not in incident[i] and e not in sel]
            cands = rng.draw_without_replacement(rng.keyed(seed, int(local_index[i]), r), eligible, n_cand)
            best = None
            for c in cands:
                M, y = fit_system(mesh, i, Ub[d], A[d], lam, q, sel + [c])
                wc, rn = scipy.optimize.nnls(M, y)
                rel = rn / np.linalg.norm(y)
                if best is None or rel < best[0] or (rel == best[0] and c < best[1]):
                    best = (rel, c, wc)
            if best is None:
                break
            res, c, w = best
            sel.append(c)
        resid[i] = res
        for s, e in enumerate(sel):
            elem[i, s] = e
            weight[i, s] = w[s]
            for a_loc, a in enumerate(mesh.tets[e]):
                da = mesh.dof_of[a]
                if da >= 0:
                    ubar[i, s, a_loc] = Ub[d][3 * da:3 * da + 3]
    return Cubature(elem, weight, ubar, resid)
