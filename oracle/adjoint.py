"""Adjoint of one implicit-Euler step (not in the paper; implicit-function theorem on
Eq. 1's optimality condition g(x*; x_t, v_t, E) = 0).

With L a function of x_{t+1} = x* and v_{t+1} = (x* - x_t)/h, and gbar = dL/dx* + dL/dv/h:
    H(x*) lam = gbar          over free DOFs, H the exact Hessian of E at x*
    dL/dx_t  = (M/h^2) lam - dL/dv / h              (free vertices; z depends on x_t)
    dL/dx_t  = dL/dx_{t+1} - (H_pf lam)             (pinned vertices: x_{t+1} = x_t there)
    dL/dv_t  = (M/h) lam                            (free vertices; 0 for pinned)
    dL/dE_e  = -sum_{a in e} lam_a . (V_e P(F_e) b_a) / E_e
               (P is linear in (mu, lam') and both are proportional to E at fixed nu)
Dense FP64; small meshes only. No contact (the barrier is left out of the adjoint).

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np

from . import fem


def step_adjoint(mesh: fem.Mesh, x_t, v_t, x1, gx1, gv1, h):
    """Returns (gx_t (V,3), gv_t (V,3), gE (T,)) for loss gradients gx1, gv1 at x1."""
    V = mesh.V
    gbar = gx1 + gv1 / h
    H = fem.global_hessian(mesh, x1, h, psd=False, dense=True)
    lam_f = np.linalg.solve(H, gbar[mesh.free].reshape(-1))
    lam = np.zeros((V, 3))
    lam[mesh.free] = lam_f.reshape(-1, 3)
    gx = np.zeros((V, 3))
    gv = np.zeros((V, 3))
    m = mesh.mass[:, None]
    gx[mesh.free] = (m / h ** 2 * lam - gv1 / h)[mesh.free]
    gv[mesh.free] = (m / h * lam)[mesh.free]
    # pinned: x_{t+1} = x_t there, and the free equilibrium couples through elastic blocks
    pin = np.nonzero(mesh.pinned)[0]
    if len(pin):
        He = fem.element_hessians(mesh, x1, h, psd=False, inertia=False)   # (T,12,12)
        coup = np.zeros((V, 3))
        lam_e = lam[mesh.tets].reshape(-1, 12)                           # lam = 0 at pinned corners
        contrib = np.einsum("tij,tj->ti", He, lam_e).reshape(-1, 4, 3)
        np.add.at(coup, mesh.tets.ravel(), contrib.reshape(-1, 3))
        gx[pin] = gx1[pin] - coup[pin]
    F = fem.deformation_gradient(mesh, x1)
    P = fem.snh_P(F, mesh.mu, mesh.lp)
    ge = mesh.vol[:, None, None] * np.einsum("tij,taj->tai", P, mesh.b)   # (T,4,3)
    gE = -np.einsum("tai,tai->t", lam[mesh.tets], ge) / mesh.youngs
    return gx, gv, gE
