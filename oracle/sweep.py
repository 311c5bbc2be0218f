"""The JGS2 Jacobi sweep and the time-step driver (Secs. 3-5, 8.1).

Per sweep k, from x^k only (Jacobi, Sec. 8.1: all vertex sub-problems at once, N_i = 3):
  g_i, H_ii    gradient and diagonal 3x3 block of E at x^k (Eq. reduced_local terms)
  R_v          polar factor (det +1) of the volume-weighted mean deformation gradient of
               the tets around v (Sec. 4.3; reading R5)
  U_{i,a}      = R_a U_bar_{i,a} R_i^T                                   (Eq. tilde_phi)
  H~_i         = sum_s w_s [U_i]_s^T H_hat_{e_s}(x^k) [U_i]_s             (Eq. cubature)
  g~_i         = sum_s w_s sum_{a in e_s} U_{i,a}^T g_a(x^k)   (reading R3 "asm": the
               assembled gradient at the element's vertices, so g~ -> 0 at equilibrium)
  (H_ii + H~_i) d_i = -(g_i + g~_i)                                      (Eq. reduced_local)
  x_i^{k+1} = x_i^k + d_i
If H_ii + H~_i fails a Cholesky test the vertex takes the uncorrected step -H_ii^{-1} g_i
(reading R7; H_ii itself is always positive definite for this material, see fem.py).

Globalisation (reading R17): the per-vertex updates form a direction D; with line search
on, x^{k+1} = x^k + alpha d with Armijo backtracking on the global energy over alpha = 2^-j,
first along D, then along the uncorrected direction D_J (always a descent direction).
Without it (the paper's plain Jacobi), x^{k+1} = x^k + D.

Stopping (reading R9): r_k = |g(x^k)| / |g(x^0)| over free DOFs; stop at the first k with
r_k <= rel_tol (returning x^k after k sweeps) or at max_sweeps. Optionally also Sec. 8's
check: the paper normalises a scene into a unit cube and stops when the positions change by
less than a tolerance between two consecutive iterations; read here as the 2-norm over all
free DOFs, |x^k - x^{k-1}| <= dx_tol * L (k >= 1), L the normalising length (default: the
largest extent of the rest positions' bounding box), tested after the residual test.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem


def polar_rotation(F):
    """Rotation closest to F (det +1): U diag(1,1,det(U V^T)) V^T from the SVD."""
    U, _, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    D = np.ones(F.shape[:-2] + (3,))
    D[..., 2] = d
    return np.einsum("...ik,...k,...kj->...ij", U, D, Vt)


def vertex_rotations(mesh: fem.Mesh, x):
    """R_v = polar(F_v), F_v = sum_{e ni v} V_e F_e / sum_{e ni v} V_e (reading R5)."""
    F = fem.deformation_gradient(mesh, x)
    Fv = np.zeros((mesh.V, 3, 3))
    wv = np.zeros(mesh.V)
    for a in range(4):
        np.add.at(Fv, mesh.tets[:, a], mesh.vol[:, None, None] * F)
        np.add.at(wv, mesh.tets[:, a], mesh.vol)
    Fv /= np.maximum(wv, 1e-300)[:, None, None]
    return polar_rotation(Fv)


@dataclass
class SweepStats:
    fallback: int = 0
    ls_rejects: int = 0


def element_gradients(mesh: fem.Mesh, x, z, h):
    """Own gradient of E_hat_e per element corner (T,4,3): V_e P b_a + m_e/h^2 (x_a - z_a),
    zero at pinned corners (the literal per-element term of Eq. cubature, reading "elem")."""
    F = fem.deformation_gradient(mesh, x)
    P = fem.snh_P(F, mesh.mu, mesh.lp)
    ge = mesh.vol[:, None, None] * np.einsum("tij,taj->tai", P, mesh.b)
    ge = ge + (mesh.rho * mesh.vol / 4.0 / h ** 2)[:, None, None] * (x - z)[mesh.tets]
    ge[mesh.pinned[mesh.tets]] = 0.0
    return ge


def correction_terms(mesh: fem.Mesh, x, g, h, cub, R, psd=False, grad="asm", z=None):
    """H~_i and g~_i of Eq. cubature for every vertex (zero for pinned / empty records)."""
    He = fem.element_hessians(mesh, x, h, psd=psd, inertia=True)
    ge = element_gradients(mesh, x, z, h) if grad == "elem" else None
    V = mesh.V
    Ht = np.zeros((V, 3, 3))
    gt = np.zeros((V, 3))
    for s in range(cub.n_cub):
        e = cub.elem[:, s]
        ok = (e >= 0) & ~mesh.pinned
        if not ok.any():
            continue
        idx = np.nonzero(ok)[0]
        es = e[ok]
        corners = mesh.tets[es]                                   # (n,4)
        Ra = R[corners]                                           # (n,4,3,3)
        Ri = R[idx]                                               # (n,3,3)
        U = np.einsum("naij,najk,nlk->nail", Ra, cub.ubar[idx, s], Ri)   # R_a Ub R_i^T
        U12 = U.reshape(len(idx), 12, 3)
        w = cub.weight[idx, s]
        Ht[idx] += w[:, None, None] * np.einsum("npi,npq,nqj->nij", U12, He[es], U12)
        ga = g[corners] if grad == "asm" else ge[es]              # (n,4,3)
        gt[idx] += w[:, None] * np.einsum("naji,naj->ni", U, ga)
    return Ht, gt


def coupled_local_terms(mesh: fem.Mesh, x, g, Hd):
    """Contact-aware local terms (Sec. 7; reading R24): a vertex i in contact with another
    body moves, in its sub-problem, together with the colliding vertices of that body (the
    same perturbation as i). With P(i) the vertices on other bodies that share an active pair
    (d < dhat) with i, free, and S_i = {i} + P(i):
      g_i' = g_i^e + sum_{b in P(i)} g_b^e + sum_{pairs l of i} kappa B'(d_l) J_S,l
      H_i' = H_ii^e + sum_{b in P(i)} H_bb^e + sum_{pairs l of i} kappa B''(d_l) J_S,l J_S,l^T
    where ^e drops the contact terms (elastic and inertial parts only; vertex i's own wall friction
    stays in its g_i^e, H_ii^e) and J_S,l is the sum of
    the pair's distance gradients over its vertices in S_i (zero for a vertex-face pair whose
    face lies on the other body: the pair moves rigidly in the sub-problem). The partners'
    other pairs and the elastic coupling between partners are left out. Returns {i: (g_i',
    H_i')} for the vertices with a cross-body pair; the others keep (g_i, H_ii)."""
    con = mesh.contact
    act = con.pairs(x, con.dhat)
    gb, Hb = con.vertex_terms(x, act, mesh.V)
    gf, Hf = con.friction_terms(x, mesh.V)
    ge, He = g - gb, Hd - Hb  # vertex i keeps its own wall friction (R25)
    body = mesh.body_of_vertex
    geo = {}
    by_vertex = {}
    for pr in act:
        d, J = con.pair_geometry(x, pr)
        geo[pr[:3]] = (d, J)
        for v, _ in J:
            by_vertex.setdefault(v, []).append(pr[:3])
    out = {}
    for i in mesh.free:
        prs = by_vertex.get(int(i), [])
        P = sorted({v for key in prs for v, _ in geo[key][1]
                    if body[v] != body[i] and not mesh.pinned[v]})
        if not P:
            continue
        S = set(P) | {int(i)}
        gi, Hi = ge[i].copy(), He[i].copy()
        for key in prs:
            d, J = geo[key]
            JS = sum((jv for v, jv in J if v in S), np.zeros(3))
            b1 = con.kappa * float(con.e1(np.array([d]), con.dhat)[0])
            b2 = con.kappa * float(con.e2(np.array([d]), con.dhat)[0])
            gi += b1 * JS
            Hi += b2 * np.outer(JS, JS)
        for b in P:  # partners: elastic and inertial parts only (their friction left out)
            gi += ge[b] - gf[b]
            Hi += He[b] - Hf[b]
        out[int(i)] = (gi, Hi)
    return out


def direction(mesh: fem.Mesh, x, z, h, cub=None, psd=False, grad="asm", stats=None, coupled=False):
    """JGS2 direction D (x^{k+1} = x^k + D without line search), the uncorrected per-vertex
    Newton direction D_J = -H_ii^{-1} g_i, and the gradient at x^k. cub=None: D = D_J.
    coupled: with contact on, D takes the contact-aware local terms of coupled_local_terms."""
    g = fem.vertex_gradient(mesh, x, z, h)
    Hd = fem.vertex_diag_blocks(mesh, x, h)
    if cub is not None:
        R = vertex_rotations(mesh, x)
        Ht, gt = correction_terms(mesh, x, g, h, cub, R, psd, grad, z)
    else:
        Ht = np.zeros_like(Hd)
        gt = np.zeros_like(g)
    cpl = coupled_local_terms(mesh, x, g, Hd) if (coupled and mesh.contact is not None) else {}
    D = np.zeros_like(x)
    DJ = np.zeros_like(x)
    for i in mesh.free:
        LJ = np.linalg.cholesky(Hd[i])
        DJ[i] = np.linalg.solve(LJ.T, np.linalg.solve(LJ, -g[i]))
        gi, Hi = cpl.get(int(i), (g[i], Hd[i]))
        try:
            L = np.linalg.cholesky(Hi + Ht[i])
            D[i] = np.linalg.solve(L.T, np.linalg.solve(L, -(gi + gt[i])))
        except np.linalg.LinAlgError:
            D[i] = DJ[i]
            if stats is not None:
                stats.fallback += 1
    if mesh.contact is not None:
        # step truncation (reading R11): |delta_v| <= 0.45 min(r_c, d_min,v)
        cand = mesh.contact.pairs(x, mesh.rc)
        lim = mesh.contact.step_limits(x, cand, mesh.rc, mesh.V)
        for arr in (D, DJ):
            nrm = np.linalg.norm(arr, axis=1)
            sc = np.where(nrm > lim, lim / np.maximum(nrm, 1e-300), 1.0)
            arr *= sc[:, None]
    return D, DJ, g


def sweep(mesh: fem.Mesh, x, z, h, cub=None, psd=False, stats=None, grad="asm"):
    """One Jacobi sweep without line search: x^{k+1} = x^k + D."""
    D, _, _ = direction(mesh, x, z, h, cub, psd, grad, stats)
    return x + D


LS_TRIALS = 8
ARMIJO_C = 1e-4


def line_search(mesh: fem.Mesh, x, z, h, D, DJ, g, stats=None):
    """Global backtracking on E (reading R17). Trials in order: the JGS2 direction D with
    alpha_j = 2^-j (j < 8), then the uncorrected direction D_J with the same alphas; the
    first trial with E(x + a d) - E(x) <= 1e-4 a g.d is taken (energy changes from
    fem.energy_change, free of cancellation). If none passes the sweep does not move
    (counted). Returns the step a*d."""
    alphas = [1.0 / (1 << j) for j in range(LS_TRIALS)]
    cand = mesh.contact.pairs(x, mesh.rc) if mesh.contact is not None else None
    for d in (D, DJ):
        slope = float(np.sum(g * d))
        dE = fem.energy_change(mesh, x, z, h, d, alphas)
        if cand is not None:
            # barrier change over the candidate pairs (truncation keeps every other pair
            # outside dhat along the whole trial segment), plus the friction change (R25)
            B0 = mesh.contact.energy(x, cand) + mesh.contact.friction_energy(x)
            dE = [de + mesh.contact.energy(x + a * d, cand) + mesh.contact.friction_energy(x + a * d) - B0
                  for a, de in zip(alphas, dE)]
        for a, de in zip(alphas, dE):
            if de <= ARMIJO_C * a * slope:
                return a * d
    if stats is not None:
        stats.ls_rejects += 1
    return np.zeros_like(D)


@dataclass
class StepResult:
    x: np.ndarray
    v: np.ndarray
    sweeps: int
    residuals: list = field(default_factory=list)
    fallback: int = 0
    ls_rejects: int = 0
    converged: bool = False
    stopped_dx: bool = False


def residual_norm(mesh, x, z, h):
    return float(np.linalg.norm(fem.vertex_gradient(mesh, x, z, h)[mesh.free]))


def run_sweeps(mesh: fem.Mesh, x, z, h, cub=None, n=1, psd=False, grad="asm", line_search_on=True,
               coupled=False):
    """Exactly n sweeps from x (no convergence test)."""
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(n):
        D, DJ, g = direction(mesh, x, z, h, cub, psd, grad, coupled=coupled)
        x = x + (line_search(mesh, x, z, h, D, DJ, g) if line_search_on else D)
    return x


def step(mesh: fem.Mesh, x_t, v_t, h, gravity, cub=None, rel_tol=1e-4, max_sweeps=100,
         psd=False, grad="asm", line_search_on=True, record_x=False, dx_tol=0.0, length_scale=0.0,
         coupled=False):
    """One implicit-Euler step (Sec. 3) solved by JGS2 sweeps from x^0 = x_t (reading R8).

    Sweep k computes g(x^k); r_k = |g(x^k)|/|g(x^0)|; the step stops at the first k with
    r_k <= rel_tol, or (dx_tol > 0, k >= 1) |x^k - x^{k-1}| <= dx_tol L, or k = max_sweeps,
    and returns x^k (k sweeps applied)."""
    z = fem.inertia_target(x_t, v_t, h, gravity)
    x = np.array(x_t, dtype=np.float64, copy=True)
    if mesh.contact is not None:
        mesh.contact.lag_friction(x_t, h)  # lagged normal forces of this step (R25)
    L = length_scale if length_scale > 0 else float(np.max(mesh.X.max(axis=0) - mesh.X.min(axis=0)))
    stats = SweepStats()
    res = []
    xs = [] if record_x else None
    g0 = None
    k = 0
    conv = False
    stop_dx = False
    dx_last = None
    while True:
        D, DJ, g = direction(mesh, x, z, h, cub, psd, grad, stats, coupled)
        gn = float(np.linalg.norm(g[mesh.free]))
        if g0 is None:
            g0 = gn
        r = gn / g0 if g0 > 0 else 0.0
        res.append(r)
        if record_x:
            xs.append(x.copy())
        if r <= rel_tol or g0 == 0.0:
            conv = True
            break
        if dx_tol > 0 and dx_last is not None and dx_last <= dx_tol * L:
            stop_dx = True
            break
        if k >= max_sweeps:
            break
        step_k = line_search(mesh, x, z, h, D, DJ, g, stats) if line_search_on else D
        dx_last = float(np.linalg.norm(step_k[mesh.free]))
        x = x + step_k
        k += 1
    out = StepResult(x, (x - x_t) / h, k, res, stats.fallback, stats.ls_rejects, conv, stop_dx)
    if record_x:
        out.xs = xs
    return out
