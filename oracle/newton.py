"""Full-space references: projected Newton (Sec. 8.3, Eq. newton_system) and the
exact dynamic subspace of Secs. 4.1-4.2 used to check the optimality theorem.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


def newton_solve(mesh: fem.Mesh, x_t, v_t, h, gravity, rel_tol=1e-11, max_iter=60, psd=True):
    """Projected Newton with backtracking Armijo (c = 1e-4, alpha halved) from x_t.

    Each iteration solves H_psd dx = -g with a sparse direct solver (library LU) over the
    free DOFs (Eq. newton_system). Stops at |g| <= rel_tol |g(x_t)| or when the energy
    can no longer decrease. Returns (x*, iterations, residual history).
    """
    z = fem.inertia_target(x_t, v_t, h, gravity)
    x = np.array(x_t, dtype=np.float64, copy=True)
    g = fem.vertex_gradient(mesh, x, z, h)
    g0 = np.linalg.norm(g[mesh.free])
    hist = [1.0]
    if g0 == 0:
        return x, 0, hist
    it = 0
    for it in range(1, max_iter + 1):
        H = fem.global_hessian(mesh, x, h, psd=psd, dense=False)
        dx = spla.spsolve(H, -fem.free_vector(mesh, g))
        D = np.zeros_like(x)
        D[mesh.free] = dx.reshape(-1, 3)
        E0 = fem.energy(mesh, x, z, h)
        slope = float(np.sum(g * D))
        alpha = 1.0
        while alpha > 1e-8:
            xn = x + alpha * D
            if fem.energy(mesh, xn, z, h) <= E0 + 1e-4 * alpha * slope:
                break
            alpha *= 0.5
        else:
            xn = x + alpha * D
        x = xn
        g = fem.vertex_gradient(mesh, x, z, h)
        r = np.linalg.norm(g[mesh.free]) / g0
        hist.append(r)
        if r <= rel_tol or (len(hist) > 3 and r >= hist[-2] * 0.999 and r < 1e-8):
            break
    return x, it, hist


def exact_subspace_step(mesh: fem.Mesh, x, z, h, psd=False):
    """One Jacobi sweep with the exact per-vertex subspace of Eq. phi at x (Sec. 4.1):
    U_C = -H_CC^{-1} H_iC^T and d_i = -(H_ii + H_iC U_C)^{-1} (g_i + U_C^T g_C), i.e.
    Eq. local_newton with Eq. relation substituted. Dense; tiny meshes only."""
    H = fem.global_hessian(mesh, x, h, psd=psd, dense=True)
    g = fem.free_vector(mesh, fem.vertex_gradient(mesh, x, z, h))
    n = H.shape[0]
    out = x.copy()
    for d, v in enumerate(mesh.free):
        I = np.arange(3 * d, 3 * d + 3)
        C = np.setdiff1d(np.arange(n), I)
        HiC = H[np.ix_(I, C)]
        UC = -np.linalg.solve(H[np.ix_(C, C)], HiC.T)
        A = H[np.ix_(I, I)] + HiC @ UC
        out[v] = x[v] - np.linalg.solve(A, g[I] + UC.T @ g[C])
    return out


def newton_step_dense(mesh: fem.Mesh, x, z, h, psd=False):
    """x + dx* with H dx* = -g (Eq. newton_system), dense."""
    H = fem.global_hessian(mesh, x, h, psd=psd, dense=True)
    g = fem.free_vector(mesh, fem.vertex_gradient(mesh, x, z, h))
    out = x.copy()
    out[mesh.free] += np.linalg.solve(H, -g).reshape(-1, 3)
    return out
