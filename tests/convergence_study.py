"""Convergence study of the readings of JGS2's correction (Secs. 3-5, 8.2-8.3, 9).

TEST INFRASTRUCTURE: built on the FP64 oracle; tests/test_convergence_study.py asserts its
findings and `python tests/convergence_study.py` prints the full table.

The paper's claim (Sec. 4.2's optimality theorem, Sec. 8.2-8.3's iteration counts) is that
the corrected Jacobi sweep converges at close to Newton's rate. The theorem holds for the
exact subspace: with U_i = [I; U_C] and the exact sums over every complement vertex,
    (U_i^T H U_i) d_i = -U_i^T g      (U_i^T H U_i = H_ii + H_iC U_C, the Schur complement)
gives d_i = (H^{-1}(-g))_i, one Newton step. The method replaces the exact sums by the
cubature of Eq. cubature: four weighted elements per vertex, trained on low eigenvectors
of the rest Hessian (Eq. cubature_weight). The readings compared here differ in what the
local matrix is, what the sampled gradient term is, how the weights are trained and how
the iteration is globalised:

  local matrix    "cub"    H_ii + H~_i, H~_i the cubature sum of Eq. cubature (the build's
                           default); "schur" the co-rotated rest Schur complement
                           R_i A_i^{-1} R_i^T, the matrix Eq. local_newton gives once Eq.
                           relation is substituted (A_i = (H_bar^{-1})_ii)
  gradient        "asm"    sum_s w_s sum_{a in e_s} U_{i,a}^T g_a with the assembled g (the
                           build's default); "elem" the element's own gradient (literal
                           Eq. cubature); "exact" the full complement sum
                           sum_{a != i} U_{i,a}^T g_a (the O(N) per vertex cost Sec. 5 avoids);
                           "none" no gradient term (H~ as a pure damper)
  training        n_train lowest eigenvectors (4, 8, 20), n_cub elements (4, 6), candidates
                  from a 256-element pool or from the whole body (the paper's draw)
  globalisation   "global" Armijo on E every sweep (reading R17); "global/k" only every k-th
                  sweep (Sec. 3 advises using the global line search sparingly);
                  "local" backtracking per vertex on its own sub-problem energy (Sec. 9: a
                  line search per sub-problem, all in parallel); "none" the plain sweep

Two measurements:
  linear    at the rest state (R = I) the sweep is the linear iteration
            e <- (I - P H_bar) e; its spectral radius rho says whether the plain sweep
            converges (rho < 1) and how fast (sweeps per decade ~ -1/log10 rho). For a
            reading whose operator has rho > 1 no fixed damping factor helps either when
            P H_bar has eigenvalues with negative real part (directions that are not descent
            directions): min over omega of rho(I - omega P H_bar) is reported.
  nonlinear sweeps of one time step to a relative residual of 1e-4 (reading R9) against
            projected Newton's iterations, on the 384-tet cube (the 5x5x5 cube scene), a
            stiff clamped beam (21x6x6 vertices, E = 1e7, the stiff beam scene's recipe)
            and a stiff free sphere (6 cells across, E = 2e6, falling with v0 = (0.3, 0, -1)).
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from oracle import fem, newton, precompute, sweep  # noqa: E402

# ------------------------------------------------------------------ scenes of the study


def cube():
    return scenes.cube_scene()


def stiff_beam():
    """The stiff beam's recipe (E = 1e7, nu = 0.45, x = 0 clamped, v0 ~ N(0, 0.05)) at
    21x6x6 vertices over 0.1 x 0.025 x 0.025 m."""
    return scenes.beam_scene(21, 6, 6, 0.1, 0.025, 1e7, 0.45, 0.05, seed=0)


def stiff_sphere():
    """A free voxel sphere (r = 0.1 m, 6 cells across: 251 vertices, 816 tets), E = 2e6,
    falling with v0 = (0.3, 0, -1) m/s, no contact."""
    X, tets = scenes.voxel_sphere(0.1, 6, center=(0.5, 0.5, 1.0))
    T = len(tets)
    v0 = np.tile([0.3, 0.0, -1.0], (len(X), 1))
    return scenes.Scene("sphere", X, tets, np.full(T, 2e6), np.full(T, 0.4), np.full(T, 1000.0),
                        np.zeros(len(X), np.uint8), v0)


def mesh_of(s):
    return fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)


# ------------------------------------------------------------------ linearised iteration


def _blockdiag_inv(blocks):
    n = 3 * len(blocks)
    out = np.zeros((n, n))
    for d, B in enumerate(blocks):
        out[3 * d:3 * d + 3, 3 * d:3 * d + 3] = np.linalg.inv(B)
    return out


def linear_operators(m, h, cub, Hbar=None):
    """Maps of one sweep at the rest state (R = I), over free DOFs:
    Hd[d] = H_ii, Ht[d] = cubature H~_i, Ainv[d] = A_i^{-1} (Schur complement),
    C_asm (g~ = C_asm g), C_elem (linear part of the element-gradient term: g~ = C_elem (x - X)
    + const), C_exact (g~ = full complement sum)."""
    if Hbar is None:
        Hbar = precompute.rest_hessian(m, h)
    N = Hbar.shape[0]
    nf = N // 3
    Ub, A = precompute.ubar_all(m, Hbar)
    He = fem.element_hessians(m, m.X, h, psd=False, inertia=True)
    Hd = np.array([Hbar[3 * d:3 * d + 3, 3 * d:3 * d + 3] for d in range(nf)])
    Ht = np.zeros((nf, 3, 3))
    C_asm = np.zeros((N, N))
    C_elem = np.zeros((N, N))
    for i in m.free:
        d = m.dof_of[i]
        for s in range(cub.n_cub):
            e = cub.elem[i, s]
            if e < 0:
                continue
            w = cub.weight[i, s]
            U12 = cub.ubar[i, s].reshape(12, 3)
            Ht[d] += w * U12.T @ He[e] @ U12
            dofs = [m.dof_of[a] for a in m.tets[e]]
            for al, da in enumerate(dofs):
                if da < 0:
                    continue
                C_asm[3 * d:3 * d + 3, 3 * da:3 * da + 3] += w * cub.ubar[i, s, al].T
            # element gradient is linear in the element's corner displacements at rest:
            # g_e = He_e (x_e - X_e) + const (pinned corners fixed)
            UtH = w * U12.T @ He[e]                       # (3, 12)
            for al, da in enumerate(dofs):
                if da < 0:
                    continue
                C_elem[3 * d:3 * d + 3, 3 * da:3 * da + 3] += UtH[:, 3 * al:3 * al + 3]
    C_exact = np.zeros((N, N))
    for d in range(nf):
        C_exact[3 * d:3 * d + 3] = Ub[d].T
        C_exact[3 * d:3 * d + 3, 3 * d:3 * d + 3] -= np.eye(3)
    Ainv = np.array([np.linalg.inv(A[d]) for d in range(nf)])
    return dict(H=Hbar, Hd=Hd, Ht=Ht, Ainv=Ainv, C_asm=C_asm, C_elem=C_elem, C_exact=C_exact)


def iteration_matrix(ops, local="cub", grad="asm"):
    """Error propagation of the plain sweep at rest: e <- (I - P) e with
    P = M^{-1} (H + C H) for gradient terms applied to the assembled gradient (asm, exact)
    or M^{-1} (H + C_elem) for the element gradient; M = blockdiag of the local matrix."""
    H = ops["H"]
    if local == "cub":
        Minv = _blockdiag_inv(ops["Hd"] + ops["Ht"])
    elif local == "jacobi":
        Minv = _blockdiag_inv(ops["Hd"])
    elif local == "schur":
        Minv = _blockdiag_inv(ops["Ainv"])
    else:
        raise ValueError(local)
    if grad == "none":
        PH = Minv @ H
    elif grad == "elem":
        PH = Minv @ (H + ops["C_elem"])
    else:
        PH = Minv @ (H + ops["C_" + grad] @ H)
    return np.eye(H.shape[0]) - PH, PH


def spectral_summary(ops, local, grad):
    """(rho, min Re eig(PH), best damped rho over omega in (0, 1.5])."""
    Mi, PH = iteration_matrix(ops, local, grad)
    ev = np.linalg.eigvals(PH)
    rho = float(np.abs(1.0 - ev).max())
    best = min(float(np.abs(1.0 - w * ev).max()) for w in np.linspace(0.02, 1.5, 75))
    return rho, float(ev.real.min()), best


# ------------------------------------------------------------------ nonlinear step


def local_energies(m, x, z, h, d, alphas):
    """Sub-problem energy change per free vertex i along its own update alone:
    E_i(x_i + a d_i) - E_i(x_i), with E_i = m_i/(2h^2)|x_i - z_i|^2 + the elastic energy of the
    tets around i (the other vertices held; Sec. 3's sub-problem E_i). (len(alphas), V)."""
    F = fem.deformation_gradient(m, x)
    psi0 = fem.snh_psi(F, m.mu, m.lp)
    out = np.zeros((len(alphas), m.V))
    for k, a in enumerate(alphas):
        acc = np.zeros(m.V)
        for c in range(4):
            v = m.tets[:, c]
            Fa = F + a * np.einsum("ti,tj->tij", d[v], m.b[:, c, :])
            np.add.at(acc, v, m.vol * (fem.snh_psi(Fa, m.mu, m.lp) - psi0))
        dx = (x - z)
        acc += 0.5 * m.mass / h ** 2 * (2 * a * np.sum(d * dx, axis=1) + a * a * np.sum(d * d, axis=1))
        out[k] = acc
    return out


def corrected_direction(m, x, z, h, cub, local="cub", grad="asm", A=None, Ub=None):
    """Per-vertex direction of one sweep and the local model's terms (gt, Ht). A: the
    A_i = (H_bar^{-1})_ii blocks (local = "schur"); Ub: every U_bar_i (grad = "exact")."""
    g = fem.vertex_gradient(m, x, z, h)
    Hd = fem.vertex_diag_blocks(m, x, h)
    Ht = np.zeros_like(Hd)
    gt = np.zeros_like(g)
    R = sweep.vertex_rotations(m, x)
    if cub is not None and grad != "exact":
        Ht, gt = sweep.correction_terms(m, x, g, h, cub, R, False, "elem" if grad == "elem" else "asm", z)
        if grad == "none":
            gt[:] = 0.0
    if grad == "exact":
        gf = g[m.free]
        for d, i in enumerate(m.free):
            # sum over complement vertices a of R_a Ub_{i,a} R_i^T, transposed, times g_a
            U = Ub[d].reshape(-1, 3, 3)
            Ua = np.einsum("aij,ajk,lk->ail", R[m.free], U, R[i])
            Ua[d] = 0.0
            gt[i] = np.einsum("aji,aj->i", Ua, gf)
        if cub is not None:
            Ht, _ = sweep.correction_terms(m, x, g, h, cub, R, False, "asm", z)
    D = np.zeros_like(x)
    for d, i in enumerate(m.free):
        if local == "schur":
            M = R[i] @ np.linalg.inv(A[d]) @ R[i].T
        elif local == "jacobi":
            M = Hd[i]
        else:
            M = Hd[i] + Ht[i]
        try:
            L = np.linalg.cholesky(M)
            D[i] = np.linalg.solve(L.T, np.linalg.solve(L, -(g[i] + gt[i])))
        except np.linalg.LinAlgError:
            D[i] = np.linalg.solve(Hd[i], -g[i])
    return D, g, gt, Ht


def run_step(s, cub=None, local="cub", grad="asm", globalise="global", every=4, max_sweeps=400,
             rel_tol=1e-4, m=None, A=None, Ub=None):
    """Sweeps of one time step from x_t to r <= rel_tol (or the cap, or divergence past
    r = 1e6). Returns (sweeps, final r)."""
    m = mesh_of(s) if m is None else m
    h = s.dt
    z = fem.inertia_target(s.X, s.v0, h, s.gravity)
    x = s.X.copy()
    g0 = None
    alphas = [1.0 / (1 << j) for j in range(8)]
    r = 1.0
    for k in range(max_sweeps + 1):
        D, g, gt, Ht = corrected_direction(m, x, z, h, cub, local, grad, A, Ub)
        gn = float(np.linalg.norm(g[m.free]))
        g0 = gn if g0 is None else g0
        r = gn / g0 if g0 > 0 else 0.0
        if not np.isfinite(r) or r > 1e6 or r <= rel_tol or k == max_sweeps:
            return k, r
        if globalise == "global" or (globalise == "global/k" and k % every == 0):
            DJ = np.zeros_like(x)
            Hd = fem.vertex_diag_blocks(m, x, h)
            for i in m.free:
                DJ[i] = np.linalg.solve(Hd[i], -g[i])
            x = x + sweep.line_search(m, x, z, h, D, DJ, g)
        elif globalise == "local":
            dE = local_energies(m, x, z, h, D, alphas)
            # local model of the sub-problem: its own energy plus the correction's terms
            lin = np.sum(gt * D, axis=1)
            quad = 0.5 * np.einsum("vi,vij,vj->v", D, Ht, D)
            slope = np.sum((g + gt) * D, axis=1)
            step = np.zeros(m.V)
            for a, de in reversed(list(zip(alphas, dE))):
                ok = de + a * lin + a * a * quad <= 1e-4 * a * slope
                step = np.where(ok, a, step)
            x = x + step[:, None] * D
        else:
            x = x + D
    return max_sweeps, r


def newton_iterations(s, rel_tol=1e-4):
    m = mesh_of(s)
    _, it, _ = newton.newton_solve(m, s.X, s.v0, s.dt, s.gravity, rel_tol=rel_tol)
    return it


# ------------------------------------------------------------------ table


def main():
    rows = []
    for name, mk in [("cube", cube), ("stiff beam", stiff_beam), ("stiff sphere", stiff_sphere)]:
        s = mk()
        m = mesh_of(s)
        H = precompute.rest_hessian(m, s.dt)
        Ub, A = precompute.ubar_all(m, H)
        nN = newton_iterations(s)
        cubs = {
            "nt20": precompute.train_cubature(m, s.dt, Hbar=H),
            "nt4": precompute.train_cubature(m, s.dt, n_train=4, Hbar=H),
            "nt8": precompute.train_cubature(m, s.dt, n_train=8, Hbar=H),
            "nt20 ncub6": precompute.train_cubature(m, s.dt, n_cub=6, Hbar=H),
            "nt20 whole body": precompute.train_cubature(m, s.dt, n_pool=10 ** 9, Hbar=H),
        }
        print(f"== {name}: V={m.V} T={m.T}; projected Newton: {nN} iterations to 1e-4")
        print(f"   {'reading':40s} {'rho':>9s} {'minRe':>8s} {'best w':>8s}  sweeps (r) global | global/4 | local | none")
        cases = [("jacobi", None, "jacobi", "none")]
        for key in cubs:
            cases.append((f"cub + asm, {key}", key, "cub", "asm"))
        cases += [("cub + elem, nt20", "nt20", "cub", "elem"),
                  ("cub + none (damper only), nt20", "nt20", "cub", "none"),
                  ("schur + asm, nt20", "nt20", "schur", "asm"),
                  ("cub + exact g~", "nt20", "cub", "exact"),
                  ("schur + exact g~", "nt20", "schur", "exact")]
        for label, key, local, grad in cases:
            cub = cubs[key] if key else None
            ops = linear_operators(m, s.dt, cub if cub is not None else cubs["nt20"], H)
            rho, mre, best = spectral_summary(ops, local, grad)
            res = []
            for glob in ("global", "global/k", "local", "none"):
                n, r = run_step(s, cub, local, grad, glob, m=m, A=A, Ub=Ub, max_sweeps=300)
                res.append(f"{n}({r:.1e})")
            print(f"   {label:40s} {rho:9.3g} {mre:8.3f} {best:8.3f}  " + " | ".join(res))
            rows.append((name, label, rho, mre, best, res, nN))
    return rows


if __name__ == "__main__":
    main()
