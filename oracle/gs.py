"""Gauss-Seidel parallelisation of JGS2 (Sec. 8.1), FP64, for the oracle.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it. The CUDA Gauss-Seidel step
(jgs2_step_gs) shares nothing with it.

Sec. 8.1: the vertex sub-problems are grouped by a graph colouring so that no two
vertices of a group share an element. A GS sweep solves the groups one after another,
every group at the positions its predecessors left. Each group is one generalised
sub-problem. Its subspace is precomputed for the group as a whole: the unit perturbation
of a DOF of vertex i in group G keeps the other DOFs of G fixed (the constraint of Eq. cms
applied to the whole group), so U_bar_i^G is zero at the other vertices of G.

Readings taken here (beside those of the Jacobi sweep):
  colouring   greedy over the free vertices in caller order: each takes the smallest colour
              that no earlier free vertex sharing a tet with it has (pinned vertices are no
              DOFs and constrain nothing);
  sweep       for each colour c in increasing order: the JGS2 direction of the vertices of
              colour c at the current x (the same local system as the Jacobi sweep, with
              the group's U_bar), the global Armijo line search (reading R17) along that
              restricted direction and then the restricted uncorrected direction, update;
  stopping    r_k = |g(x^k)| / |g(x^0)| at the start of each GS sweep (reading R9).
"""
from __future__ import annotations

import numpy as np
import scipy.optimize

from . import fem, rng
from .precompute import Cubature, body_eigs, body_pool
from .sweep import SweepStats, StepResult, direction, line_search


def greedy_colouring(mesh: fem.Mesh):
    """Colour per vertex (-1 for pinned): the smallest colour not taken by an earlier free
    vertex (caller order) that shares a tet with it."""
    V = mesh.V
    nbr = [set() for _ in range(V)]
    for t in mesh.tets:
        for a in t:
            for b in t:
                if a != b:
                    nbr[a].add(int(b))
    col = -np.ones(V, dtype=np.int64)
    for v in mesh.free:
        used = {int(col[u]) for u in nbr[v] if col[u] >= 0}
        c = 0
        while c in used:
            c += 1
        col[v] = c
    return col


def ubar_groups(mesh: fem.Mesh, Hbar, colour):
    """Generalised-sub-problem subspaces (Sec. 8.1 with Eq. cms): for free vertex i of group
    G, U_bar_i^G (N, 3) minimises the rest energy 1/2 u^T H_bar u subject to u_i = unit and
    u_j = 0 for the other j in G: u_C = -H_CC^{-1} H_Ci on C = the DOFs outside G. Dense;
    tiny meshes only. Returns (nf, N, 3) in free-DOF order."""
    N = Hbar.shape[0]
    nf = N // 3
    Ub = np.zeros((nf, N, 3))
    fcol = colour[mesh.free]
    for c in np.unique(fcol):
        G = np.nonzero(fcol == c)[0]
        gd = (3 * G[:, None] + np.arange(3)[None, :]).ravel()
        C = np.setdiff1d(np.arange(N), gd)
        HCC = Hbar[np.ix_(C, C)]
        for d in G:
            I = np.arange(3 * d, 3 * d + 3)
            Ub[d][I] = np.eye(3)
            if C.size:
                Ub[d][C] = -np.linalg.solve(HCC, Hbar[np.ix_(C, I)])
    return Ub


def train_cubature_gs(mesh: fem.Mesh, h, colour, n_cub=4, n_train=20, n_cand=32, n_pool=256,
                      nnls_tol=0.01, seed=0, Hbar=None):
    """Greedy NNLS cubature (Sec. 5, Eq. cubature_weight) for the generalised sub-problems:
    the Jacobi training with U_bar_i^G in place of U_bar_i. For a training pose q (an
    eigenvector of H_bar, H_bar q = lam q) the column of element e is
    sum_{a in e} U_bar_{i,a}^T (H_bar q)_a and the target is sum_{a != i} U_bar_{i,a}^T
    (H_bar q)_a = lam (U_bar_i^T q - q_i), both scaled by the target's norm (reading R3
    asm; the same seeded pools and candidate draws as the Jacobi training)."""
    if Hbar is None:
        Hbar = fem.global_hessian(mesh, mesh.X, h, psd=False, dense=True)
    Ub = ubar_groups(mesh, Hbar, colour)
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

    def system(d, lam, q, elems):
        b = lam[:, None] * (q @ Ub[d] - q[:, 3 * d:3 * d + 3])
        nb = np.linalg.norm(b, axis=1)
        keep = nb > 1e-12 * max(nb.max(), 1e-300)
        cols = []
        for e in elems:
            c = np.zeros_like(b)
            for a in mesh.tets[e]:
                da = mesh.dof_of[a]
                if da >= 0:
                    c += lam[:, None] * (q[:, 3 * da:3 * da + 3] @ Ub[d][3 * da:3 * da + 3])
            cols.append((c[keep] / nb[keep, None]).ravel())
        y = (b[keep] / nb[keep, None]).ravel()
        return (np.array(cols).T if cols else np.zeros((y.size, 0))), y

    for i in mesh.free:
        d = mesh.dof_of[i]
        lam, q = eig[mesh.body_of_vertex[i]]
        sel, w, res = [], np.zeros(0), 1.0
        for r in range(n_cub):
            if res < nnls_tol:
                break
            eligible = [e for e in pools[mesh.body_of_vertex[i]] if e not in incident[i] and e not in sel]
            cands = rng.draw_without_replacement(rng.keyed(seed, int(local_index[i]), r), eligible, n_cand)
            best = None
            for c in cands:
                M, y = system(d, lam, q, sel + [c])
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


def gs_sweep(mesh: fem.Mesh, x, z, h, colour, cub=None, stats=None):
    """One GS sweep: the colours in increasing order, each a masked JGS2 direction at the
    current x, the line search along it (reading R17) and the update."""
    x = np.array(x, dtype=np.float64, copy=True)
    for c in range(int(colour.max()) + 1):
        D, DJ, g = direction(mesh, x, z, h, cub, stats=stats)
        m = (colour == c)[:, None]
        x = x + line_search(mesh, x, z, h, D * m, DJ * m, g, stats)
    return x


def gs_step(mesh: fem.Mesh, x_t, v_t, h, gravity, colour, cub=None, rel_tol=1e-4, max_sweeps=100):
    """One implicit-Euler step (Sec. 3) by GS sweeps from x^0 = x_t; stopping as the Jacobi
    driver (r_k at the start of each sweep)."""
    z = fem.inertia_target(x_t, v_t, h, gravity)
    x = np.array(x_t, dtype=np.float64, copy=True)
    stats = SweepStats()
    res = []
    g0 = None
    k = 0
    conv = False
    while True:
        g = fem.vertex_gradient(mesh, x, z, h)
        gn = float(np.linalg.norm(g[mesh.free]))
        g0 = gn if g0 is None else g0
        r = gn / g0 if g0 > 0 else 0.0
        res.append(r)
        if r <= rel_tol or g0 == 0.0:
            conv = True
            break
        if k >= max_sweeps:
            break
        x = gs_sweep(mesh, x, z, h, colour, cub, stats)
        k += 1
    return StepResult(x, (x - x_t) / h, k, res, stats.fallback, stats.ls_rejects, conv)
