"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it pins. A plausible slip in the oracle (dropped term, wrong
sign, transposed rotation, wrong Schur block) fails at least one of them.
"""
import numpy as np
import pytest

import scenes
from oracle import fem, local, newton, precompute, rng, sweep


@pytest.fixture(scope="module")
def cube():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return s, m


@pytest.fixture(scope="module")
def cube_cub(cube):
    s, m = cube
    return precompute.train_cubature(m, s.dt)


def deformed(s, m, scale=2e-3, seed=3):
    return scenes.perturbed_state(s.X, s.pinned, scale, seed)


# ---------------------------------------------------------------- T1: derivatives (Sec. 3)

def test_material_derivatives_fd():
    r = np.random.default_rng(0)
    for trial in range(5):
        F = np.eye(3) + 0.3 * r.normal(size=(3, 3))
        mu, lp = 2.0 + r.random(), 5.0 + r.random()
        eps = 1e-6
        P = fem.snh_P(F, mu, lp)
        A = fem.snh_dPdF(F, mu, lp)
        for k in range(9):
            dF = np.zeros(9)
            dF[k] = eps
            dF = dF.reshape(3, 3)
            dpsi = (fem.snh_psi(F + dF, mu, lp) - fem.snh_psi(F - dF, mu, lp)) / (2 * eps)
            assert abs(dpsi - P.ravel()[k]) < 1e-7 * max(1, abs(P).max())
            dP = (fem.snh_P(F + dF, mu, lp) - fem.snh_P(F - dF, mu, lp)) / (2 * eps)
            assert np.allclose(dP.ravel(), A[:, k], atol=1e-6 * max(1, abs(A).max()))
        assert np.allclose(A, A.T, atol=1e-12)


def test_energy_gradient_hessian_fd(cube):
    s, m = cube
    h = s.dt
    x = deformed(s, m)
    z = fem.inertia_target(s.X, 0.1 * np.ones_like(s.X), h, s.gravity)
    g = fem.vertex_gradient(m, x, z, h)
    H = fem.global_hessian(m, x, h)
    r = np.random.default_rng(1)
    for _ in range(3):
        d = np.zeros_like(x)
        d[m.free] = r.normal(size=(m.free.size, 3))
        eps = 1e-7
        dE = (fem.energy(m, x + eps * d, z, h) - fem.energy(m, x - eps * d, z, h)) / (2 * eps)
        assert abs(dE - np.sum(g * d)) < 1e-6 * abs(dE)
        dg = (fem.vertex_gradient(m, x + eps * d, z, h) - fem.vertex_gradient(m, x - eps * d, z, h)) / (2 * eps)
        Hd = H @ fem.free_vector(m, d)
        assert np.allclose(fem.free_vector(m, dg), Hd, atol=1e-5 * abs(Hd).max())
    assert np.allclose(H, H.T, atol=1e-9 * abs(H).max())
    # diagonal blocks used by the sweep equal the global Hessian's
    Hd = fem.vertex_diag_blocks(m, x, h)
    for d_, v in enumerate(m.free[:20]):
        assert np.allclose(Hd[v], H[3 * d_:3 * d_ + 3, 3 * d_:3 * d_ + 3], rtol=1e-12, atol=1e-9)


def test_diag_block_closed_form_is_spd(cube):
    """The det-Hessian term drops out of a vertex's diagonal block (eps_jln b_j b_l = 0),
    so H_vv = m/h^2 I + sum V(mu |b|^2 I + lam' G G^T) is positive definite even for
    inverted elements."""
    s, m = cube
    x = scenes.perturbed_state(s.X, s.pinned, 0.02, seed=9)  # large: some tets invert
    F = fem.deformation_gradient(m, x)
    assert (np.linalg.det(F) < 0).any()
    Hd = fem.vertex_diag_blocks(m, x, s.dt)
    for v in m.free:
        G = np.zeros((3, 3))
        for t in np.nonzero(np.any(m.tets == v, axis=1))[0]:
            c = int(np.nonzero(m.tets[t] == v)[0][0])
            b = m.b[t, c]
            Gc = fem.cofactor(F[t]) @ b
            G += m.vol[t] * (m.mu[t] * (b @ b) * np.eye(3) + m.lp[t] * np.outer(Gc, Gc))
        G += m.mass[v] / s.dt ** 2 * np.eye(3)
        assert np.allclose(Hd[v], G, rtol=1e-10, atol=1e-10)
        assert np.linalg.eigvalsh(Hd[v]).min() > 0


# ---------------------------------------------------------------- T2: rest state (R1, R2)

def test_rest_state(cube):
    s, m = cube
    g = fem.vertex_gradient(m, s.X, s.X, s.dt)
    assert np.abs(g).max() < 1e-12
    mu, lp = 3.0, 11.0
    lam = lp - mu
    A = fem.snh_dPdF(np.eye(3), mu, lp)
    r = np.random.default_rng(2)
    for _ in range(4):
        dF = r.normal(size=(3, 3))
        lin = mu * (dF + dF.T) + lam * np.trace(dF) * np.eye(3)
        assert np.allclose((A @ dF.ravel()).reshape(3, 3), lin, atol=1e-12)
    w = np.linalg.eigvalsh(A)
    assert w.min() > -1e-12
    assert np.allclose(fem.psd_clamp(A), A, atol=1e-12)
    R = sweep.vertex_rotations(m, s.X)
    assert np.allclose(R, np.eye(3)[None], atol=1e-12)


# ---------------------------------------------------------------- T3: Sec. 6 identities

def test_full_coordinate_precompute_matches_cms(cube):
    s, m = cube
    H = precompute.rest_hessian(m, s.dt)
    Ub, A = precompute.ubar_all(m, H)
    n = H.shape[0]
    for d in [0, 17, 55, 99]:
        I = np.arange(3 * d, 3 * d + 3)
        C = np.setdiff1d(np.arange(n), I)
        # S_i U_bar_i = I  (constraint of Eq. cms_constraint)
        assert np.allclose(Ub[d][I], np.eye(3), atol=1e-12)
        # H_bar U_bar_i vanishes off the rows of i (Eq. cms_constraint)
        HU = H @ Ub[d]
        assert np.abs(HU[C]).max() < 1e-9 * np.abs(HU[I]).max()
        # complement rows equal U_C = -H_CC^{-1} H_iC^T of Eq. cms (direct solve)
        UC = -np.linalg.solve(H[np.ix_(C, C)], H[np.ix_(I, C)].T)
        assert np.allclose(Ub[d][C], UC, atol=1e-10 * np.abs(UC).max())
        # U_bar^T H_bar U_bar = A_i^{-1} = Schur complement H_ii - H_iC H_CC^-1 H_Ci
        schur = H[np.ix_(I, I)] - H[np.ix_(I, C)] @ np.linalg.solve(H[np.ix_(C, C)], H[np.ix_(C, I)])
        assert np.allclose(Ub[d].T @ H @ Ub[d], schur, rtol=1e-9)
        assert np.allclose(np.linalg.inv(A[d]), schur, rtol=1e-9)
        # G_i = -(S_i H^-1 S_i^T)^-1 and U_bar = -H^-1 S_i^T G_i (Eq. u)
        G = -np.linalg.inv(np.linalg.inv(H)[np.ix_(I, I)])
        assert np.allclose(Ub[d], -np.linalg.inv(H)[:, I] @ G, atol=1e-12)


def test_rest_hessian_per_body_block_diagonal():
    X1, t1 = scenes.kuhn_grid(3, 3, 3, (0.02, 0.02, 0.02))
    X = np.vstack([X1, X1 + [0.1, 0, 0]])
    t = np.vstack([t1, t1 + len(X1)]).astype(np.int32)
    T = len(t)
    m = fem.Mesh(X, t, np.full(T, 1e5), np.full(T, 0.3), np.full(T, 1e3), np.zeros(len(X), np.uint8))
    assert m.n_bodies == 2 and m.body_of_vertex[0] == 0 and m.body_of_vertex[-1] == 1
    H = precompute.rest_hessian(m, 1 / 120)
    n1 = 3 * len(X1)
    assert np.abs(H[:n1, n1:]).max() == 0.0
    # free body: H_bar is positive definite only thanks to M/h^2 (reading R2)
    assert np.linalg.eigvalsh(H).min() > 0


# ---------------------------------------------------------------- T4: optimality (Sec. 4.2)

def test_optimality_theorem_exact_subspace_equals_newton(cube):
    s, m = cube
    x = deformed(s, m, 3e-3)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    a = newton.exact_subspace_step(m, x, z, s.dt)
    b = newton.newton_step_dense(m, x, z, s.dt)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b - x).max()


# ---------------------------------------------------------------- T5: co-rotation (Eq. tilde_phi)

def test_rigid_rotation_and_translation_invariance(cube, cube_cub):
    s, m = cube
    x = deformed(s, m, 2e-3, seed=5)
    z = fem.inertia_target(s.X, 0.05 * np.ones_like(s.X), s.dt, s.gravity)
    D, DJ, _ = sweep.direction(m, x, z, s.dt, cube_cub)
    q = np.array([0.3, -0.5, 0.8])
    q /= np.linalg.norm(q)
    K = np.array([[0, -q[2], q[1]], [q[2], 0, -q[0]], [-q[1], q[0], 0]])
    Q = np.eye(3) + np.sin(0.7) * K + (1 - np.cos(0.7)) * K @ K
    Dq, DJq, _ = sweep.direction(m, x @ Q.T, z @ Q.T, s.dt, cube_cub)
    assert np.allclose(Dq, D @ Q.T, atol=1e-9 * np.abs(D).max())
    assert np.allclose(DJq, DJ @ Q.T, atol=1e-9 * np.abs(DJ).max())
    tr = np.array([0.3, -1.0, 2.0])
    Dt, _, _ = sweep.direction(m, x + tr, z + tr, s.dt, cube_cub)
    assert np.allclose(Dt, D, atol=1e-8 * np.abs(D).max())
    R = sweep.vertex_rotations(m, x @ Q.T)
    R0 = sweep.vertex_rotations(m, x)
    assert np.allclose(R, Q[None] @ R0, atol=1e-10)


def test_polar_rotation_properties():
    r = np.random.default_rng(4)
    F = r.normal(size=(50, 3, 3))
    R = sweep.polar_rotation(F)
    assert np.allclose(R @ np.swapaxes(R, 1, 2), np.eye(3)[None], atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0)
    # R^T F is symmetric when det F > 0 (polar factor)
    pos = np.linalg.det(F) > 0
    S = np.swapaxes(R, 1, 2) @ F
    assert np.allclose(S[pos], np.swapaxes(S[pos], 1, 2), atol=1e-12)


# ---------------------------------------------------------------- T6: cubature (Sec. 5)

def test_cubature_full_sum_closed_form(cube):
    """With every element not incident to i sampled at weight 1 and x = X (R = I):
    H~_i = sum_{e not ni i} U^T H_e U = A_i^{-1} - U_bar_i^T H_loc U_bar_i, where H_loc sums
    the element Hessians around i (because H_bar U_bar_i = S_i^T A_i^{-1})."""
    s, m = cube
    h = s.dt
    Hbar = precompute.rest_hessian(m, h)
    Ub, A = precompute.ubar_all(m, Hbar)
    He = fem.element_hessians(m, s.X, h)
    for i in [m.free[3], m.free[40], m.free[77]]:
        d = m.dof_of[i]
        rem = np.nonzero(~np.any(m.tets == i, axis=1))[0]
        nc = len(rem)
        elem = -np.ones((m.V, nc), np.int64)
        elem[i] = rem
        w = np.zeros((m.V, nc))
        w[i] = 1.0
        ub = np.zeros((m.V, nc, 4, 3, 3))
        for sl, e in enumerate(rem):
            for a_loc, a in enumerate(m.tets[e]):
                if m.dof_of[a] >= 0:
                    ub[i, sl, a_loc] = Ub[d][3 * m.dof_of[a]:3 * m.dof_of[a] + 3]
        cub = precompute.Cubature(elem, w, ub, np.zeros(m.V))
        R = np.tile(np.eye(3), (m.V, 1, 1))
        Ht, _ = sweep.correction_terms(m, s.X, np.zeros_like(s.X), h, cub, R)
        inc = np.nonzero(np.any(m.tets == i, axis=1))[0]
        Hloc = np.zeros_like(Hbar)
        for e in inc:
            dofs = np.concatenate([3 * m.dof_of[a] + np.arange(3) if m.dof_of[a] >= 0 else [-1, -1, -1]
                                   for a in m.tets[e]])
            ok = dofs >= 0
            Hloc[np.ix_(dofs[ok], dofs[ok])] += He[e][np.ix_(ok, ok)]
        closed = np.linalg.inv(A[d]) - Ub[d].T @ Hloc @ Ub[d]
        assert np.allclose(Ht[i], closed, rtol=1e-8, atol=1e-8 * np.abs(closed).max())


def test_training_target_closed_form(cube):
    """b^(t) = sum_{a != i} U_bar_{i,a}^T (H_bar q_t)_a = A_i^{-1} q_{t,i} - lambda_t q_{t,i}."""
    s, m = cube
    Hbar = precompute.rest_hessian(m, s.dt)
    Ub, A = precompute.ubar_all(m, Hbar)
    lam, q = precompute.body_eigs(m, Hbar, 0, 6)
    assert np.allclose(Hbar @ q.T, q.T * lam[None], atol=1e-8 * lam.max())
    for d in [5, 60]:
        i = m.free[d]
        brute = []
        for t in range(len(lam)):
            Hq = Hbar @ q[t]
            acc = np.zeros(3)
            for dd in range(len(m.free)):
                if dd != d:
                    acc += Ub[d][3 * dd:3 * dd + 3].T @ Hq[3 * dd:3 * dd + 3]
            brute.append(acc)
        M, y = precompute.fit_system(m, i, Ub[d], A[d], lam, q, [])
        qi = q[:, 3 * d:3 * d + 3]
        closed = qi @ np.linalg.inv(A[d]).T - lam[:, None] * qi
        assert np.allclose(np.array(brute), closed, atol=1e-9 * np.abs(closed).max())


def test_greedy_cubature_properties(cube, cube_cub):
    s, m = cube
    c = cube_cub
    inc = [set(np.nonzero(np.any(m.tets == v, axis=1))[0]) for v in range(m.V)]
    for v in m.free:
        sel = [e for e in c.elem[v] if e >= 0]
        assert len(sel) >= 1 and len(set(sel)) == len(sel)
        assert not (set(sel) & inc[v])                       # remote elements (R4)
        assert (c.weight[v] >= 0).all()                       # NNLS (Eq. cubature_weight)
        assert 0.0 <= c.residual[v] <= 1.0 + 1e-12
        assert len(sel) == c.n_cub or c.residual[v] < 0.01    # stops at n_cub or tolerance
    assert (c.elem[m.pinned] == -1).all()


def test_splitmix64_draws():
    g1 = rng.keyed(7, 3, 1)
    g2 = rng.keyed(7, 3, 1)
    a = [g1.next() for _ in range(5)]
    assert a == [g2.next() for _ in range(5)]
    assert a != [rng.keyed(7, 3, 2).next() for _ in range(5)]
    picks = rng.draw_without_replacement(rng.keyed(1, 2, 3), list(range(100)), 30)
    assert len(set(picks)) == 30 and all(0 <= p < 100 for p in picks)
    # the first output of SplitMix64 from state 0 is mix(GAMMA)
    assert rng.SplitMix64(0).next() == rng.mix(rng.GAMMA)


# ---------------------------------------------------------------- T7/T8: convergence

def test_fixed_point_is_newton_minimiser(cube, cube_cub):
    s, m = cube
    xs, it, hist = newton.newton_solve(m, s.X, s.v0, s.dt, s.gravity)
    assert hist[-1] < 1e-9
    r = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cube_cub, rel_tol=1e-9, max_sweeps=2000)
    assert r.converged
    err = np.linalg.norm(r.x - xs) / np.linalg.norm(xs - s.X)
    assert err < 1e-6


def test_energy_change_matches_plain_difference(cube):
    s, m = cube
    x = deformed(s, m, 3e-3, seed=12)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    d = scenes.perturbed_state(np.zeros_like(s.X), s.pinned, 1e-3, seed=13)
    alphas = [1.0, 0.5, 0.25, 1 / 128]
    got = fem.energy_change(m, x, z, s.dt, d, alphas)
    E0 = fem.energy(m, x, z, s.dt)
    for a, dE in zip(alphas, got):
        plain = fem.energy(m, x + a * d, z, s.dt) - E0
        assert abs(dE - plain) <= 1e-9 * abs(plain) + 1e-13 * abs(E0)


def test_energy_decreases_every_sweep_with_line_search(cube, cube_cub):
    s, m = cube
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    x = s.X.copy()
    E = fem.energy(m, x, z, s.dt)
    for _ in range(15):
        x = sweep.run_sweeps(m, x, z, s.dt, cube_cub, 1)
        En = fem.energy(m, x, z, s.dt)
        assert En <= E + 1e-15 * abs(E)
        E = En


def test_local_direction_matches_global(cube, cube_cub):
    s, m = cube
    x = deformed(s, m, 2e-3, seed=11)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    D, DJ, _ = sweep.direction(m, x, z, s.dt, cube_cub)
    lm = local.LocalMesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    for i in m.free[[0, 13, 50, 99]]:
        d, dj = lm.direction(i, x, z, s.dt, cube_cub.elem[i], cube_cub.weight[i], cube_cub.ubar[i])
        assert np.allclose(d, D[i], rtol=1e-10, atol=1e-14)
        assert np.allclose(dj, DJ[i], rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------- T9/T10: contact (Sec. 7)

from oracle import contact as ct  # noqa: E402


def test_barrier_closed_form():
    dh = 1e-3
    d = np.array([dh, 2 * dh])
    assert np.all(ct.barrier(d, dh) == 0) and np.all(ct.barrier_d1(d, dh) == 0) and np.all(ct.barrier_d2(d, dh) == 0)
    # C^2 at dhat: value, slope and curvature all tend to 0 from below
    e = np.array([dh * (1 - 1e-6)])
    assert ct.barrier(e, dh)[0] < 1e-20 and abs(ct.barrier_d1(e, dh)[0]) < 1e-14 and ct.barrier_d2(e, dh)[0] < 1e-5
    # blows up at 0, FD of the derivatives
    assert ct.barrier(np.array([1e-12]), dh)[0] > 1e-6 * 20
    for x in [1e-5, 2e-4, 7e-4]:
        h = 1e-9
        fd1 = (ct.barrier(np.array([x + h]), dh)[0] - ct.barrier(np.array([x - h]), dh)[0]) / (2 * h)
        fd2 = (ct.barrier_d1(np.array([x + h]), dh)[0] - ct.barrier_d1(np.array([x - h]), dh)[0]) / (2 * h)
        assert abs(fd1 - ct.barrier_d1(np.array([x]), dh)[0]) < 1e-5 * abs(fd1)
        assert abs(fd2 - ct.barrier_d2(np.array([x]), dh)[0]) < 1e-5 * abs(fd2)
        assert ct.barrier_d2(np.array([x]), dh)[0] > 0 > ct.barrier_d1(np.array([x]), dh)[0]


def test_distances_against_dense_sampling():
    r = np.random.default_rng(5)
    for _ in range(20):
        p, a, b, c = r.normal(size=(4, 3))
        d, w = ct.point_triangle(p, a, b, c)
        uv = r.random((200000, 2))
        uv = np.where(uv.sum(1, keepdims=True) > 1, 1 - uv, uv)
        pts = a + uv[:, :1] * (b - a) + uv[:, 1:] * (c - a)
        dd = np.linalg.norm(pts - p, axis=1).min()
        res = 3 * max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / np.sqrt(2e5)  # sampling spacing
        assert d <= dd + 1e-12 and dd - d < res
        assert abs(np.linalg.norm(p - (w[0] * a + w[1] * b + w[2] * c)) - d) < 1e-12
        q0, q1 = r.normal(size=(2, 3))
        d2, s, t = ct.segment_segment(a, b, q0, q1)
        st = r.random((200000, 2))
        dd2 = np.linalg.norm(a + st[:, :1] * (b - a) - q0 - st[:, 1:] * (q1 - q0), axis=1).min()
        res2 = 3 * max(np.linalg.norm(b - a), np.linalg.norm(q1 - q0)) / np.sqrt(2e5)
        assert d2 <= dd2 + 1e-12 and dd2 - d2 < res2
        assert abs(np.linalg.norm(a + s * (b - a) - q0 - t * (q1 - q0)) - d2) < 1e-12


def test_contact_gradient_fd_and_surface():
    X, tets = scenes.kuhn_grid(3, 3, 3, (0.02, 0.02, 0.02))
    X2 = X + [0.0, 0.0, 0.0205]   # a second block just above the first
    Xa = np.vstack([X, X2])
    ta = np.vstack([tets, tets + len(X)])
    bf, be, sv = ct.surface(ta, Xa)
    assert len(bf) == 2 * 6 * 2 * 4 and len(sv) == 2 * 26   # 2 cubes x 6 sides x 2x2 cells x 2 tris
    for a, b, c in bf:   # outward: the face normal points away from the solid's centroid
        cen = Xa[:len(X)].mean(0) if a < len(X) else Xa[len(X):].mean(0)
        n = np.cross(Xa[b] - Xa[a], Xa[c] - Xa[a])
        assert n @ (Xa[a] - cen) > 0
    con = ct.Contact(ta, Xa, scenes.box_planes()[:1], 1e-3, 1e4)
    x = Xa + np.random.default_rng(3).normal(0, 1e-4, Xa.shape)
    x[:, 2] += 5e-4
    pairs = con.pairs(x, 1e-3)
    assert {p[0] for p in pairs} >= {0, 1, 2}
    g, H = con.vertex_terms(x, pairs, len(x))
    for v in np.nonzero(np.abs(g).sum(1))[0][:6]:
        for k in range(3):
            e = np.zeros_like(x)
            e[v, k] = 1e-9
            fd = (con.energy(x + e, con.pairs(x + e, 1e-3)) - con.energy(x - e, con.pairs(x - e, 1e-3))) / 2e-9
            assert abs(fd - g[v, k]) <= 1e-5 * abs(g[v]).max() + 1e-9
        assert np.linalg.eigvalsh(H[v]).min() > -1e-9


def test_penalty_closed_form():
    """Reading R23: P(d) = (dhat - d)^2 / 2 below dhat, zero above; C^1 at dhat (value and
    slope vanish there), P' = d - dhat and P'' = 1 inside, finite at d = 0; central
    differences of P and P' match P' and P''."""
    dh = 1e-3
    assert ct.penalty(np.array([dh, 2 * dh]), dh).tolist() == [0.0, 0.0]
    assert ct.penalty_d1(np.array([dh]), dh)[0] == 0.0
    assert abs(ct.penalty(np.array([0.0]), dh)[0] - 0.5 * dh * dh) < 1e-20
    for x in [1e-5, 2e-4, 7e-4]:
        h = 1e-9
        fd1 = (ct.penalty(np.array([x + h]), dh)[0] - ct.penalty(np.array([x - h]), dh)[0]) / (2 * h)
        fd2 = (ct.penalty_d1(np.array([x + h]), dh)[0] - ct.penalty_d1(np.array([x - h]), dh)[0]) / (2 * h)
        assert abs(fd1 - ct.penalty_d1(np.array([x]), dh)[0]) < 1e-6 * abs(fd1)
        assert abs(fd2 - 1.0) < 1e-6 and ct.penalty_d2(np.array([x]), dh)[0] == 1.0


def test_penalty_contact_gradient_fd():
    X, tets = scenes.kuhn_grid(3, 3, 3, (0.02, 0.02, 0.02))
    Xa = np.vstack([X, X + [0.0, 0.0, 0.0205]])
    ta = np.vstack([tets, tets + len(X)])
    con = ct.Contact(ta, Xa, scenes.box_planes()[:1], 1e-3, 1e4, use_penalty=True)
    x = Xa + np.random.default_rng(3).normal(0, 1e-4, Xa.shape)
    x[:, 2] += 5e-4
    pairs = con.pairs(x, 1e-3)
    g, H = con.vertex_terms(x, pairs, len(x))
    for v in np.nonzero(np.abs(g).sum(1))[0][:6]:
        for k in range(3):
            e = np.zeros_like(x)
            e[v, k] = 1e-9
            fd = (con.energy(x + e, con.pairs(x + e, 1e-3)) - con.energy(x - e, con.pairs(x - e, 1e-3))) / 2e-9
            assert abs(fd - g[v, k]) <= 1e-5 * abs(g[v]).max() + 1e-12
        assert np.linalg.eigvalsh(H[v]).min() > -1e-12


def _contact_mesh(s):
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return m.enable_contact(s.planes, s.dhat, s.kappa, use_penalty=s.contact == 2)


def test_contact_step_stays_intersection_free():
    for s in (scenes.drop_scene(nv=3), scenes.stack_scene()):
        m = _contact_mesh(s)
        x, v = s.X.copy(), s.v0.copy()
        for _ in range(1):
            r = sweep.step(m, x, v, s.dt, s.gravity, None, 1e-4, 150)
            x, v = r.x, r.v
            pairs = m.contact.pairs(x, 10 * s.dhat)
            assert all(p[3] > 0 for p in pairs)
            assert min(r.residuals) < 0.1   # progress; the barrier makes Jacobi slow
        assert x[:, 2].min() > 0
    assert any(p[0] == 1 for p in pairs) and any(p[0] == 2 for p in pairs)


def test_no_contact_in_range_equals_plain_sweep(cube, cube_cub):
    s, m, = cube
    mc = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned).enable_contact(
        scenes.box_planes() + [0, 0, 0, -5.0], 1e-3, 1e4)   # walls 5 m away
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    a = sweep.run_sweeps(m, s.X, z, s.dt, cube_cub, 2)
    b = sweep.run_sweeps(mc, s.X, z, s.dt, cube_cub, 2)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- T11: adjoint

from oracle import adjoint  # noqa: E402


def _solve_tight(s, m, x_t, v_t):
    """Full Newton with dense solves from x_t until the residual stops decreasing."""
    z = fem.inertia_target(x_t, v_t, s.dt, s.gravity)
    x = x_t.copy()
    best = np.inf
    for _ in range(40):
        xn = newton.newton_step_dense(m, x, z, s.dt)
        r = np.linalg.norm(fem.vertex_gradient(m, xn, z, s.dt)[m.free])
        if r >= best:
            break
        x, best = xn, r
    return x


def test_adjoint_against_central_differences():
    s = scenes.small_beam_scene(5, 3, 3, E=2e5, vel_sigma=0.05, seed=2)
    T = s.n_tets
    E0 = s.youngs * np.random.default_rng(1).uniform(0.5, 1.5, T)
    mk = lambda E: fem.Mesh(s.X, s.tets, E, s.poisson, s.density, s.pinned)  # noqa: E731
    m = mk(E0)
    x_t = scenes.perturbed_state(s.X, s.pinned, 1e-4, seed=4)
    v_t = s.v0
    x1 = _solve_tight(s, m, x_t, v_t)
    r = np.random.default_rng(7)
    cx, cv = r.normal(size=x1.shape), r.normal(size=x1.shape)
    loss = lambda x1_, xt_: float(np.sum(cx * x1_) + np.sum(cv * (x1_ - xt_) / s.dt))  # noqa: E731
    gx, gv, gE = adjoint.step_adjoint(m, x_t, v_t, x1, cx, cv, s.dt)
    rel = 1e-4
    # Young's modulus of a few elements (central differences, h = 1e-4 relative)
    for e in [0, 7, T // 2, T - 1]:
        Ep, Em = E0.copy(), E0.copy()
        Ep[e] *= 1 + rel
        Em[e] *= 1 - rel
        fd = (loss(_solve_tight(s, mk(Ep), x_t, v_t), x_t) - loss(_solve_tight(s, mk(Em), x_t, v_t), x_t)) / (2 * rel * E0[e])
        assert abs(fd - gE[e]) <= 1e-4 * abs(fd) + 1e-6 * np.abs(gE).max()
    # initial state: a free and a pinned vertex component, and a velocity component
    free = np.nonzero(~s.pinned.astype(bool))[0]
    pin = np.nonzero(s.pinned.astype(bool))[0]
    for (arr_name, v, k) in [("x", free[5], 2), ("x", pin[1], 0), ("v", free[9], 1)]:
        eps = 1e-7
        if arr_name == "x":
            xp, xm = x_t.copy(), x_t.copy()
            xp[v, k] += eps
            xm[v, k] -= eps
            fd = (loss(_solve_tight(s, m, xp, v_t), xp) - loss(_solve_tight(s, m, xm, v_t), xm)) / (2 * eps)
            ref = gx[v, k]
        else:
            vp, vm = v_t.copy(), v_t.copy()
            vp[v, k] += eps
            vm[v, k] -= eps
            fd = (loss(_solve_tight(s, m, x_t, vp), x_t) - loss(_solve_tight(s, m, x_t, vm), x_t)) / (2 * eps)
            ref = gv[v, k]
        assert abs(fd - ref) <= 1e-4 * abs(fd) + 1e-7, (arr_name, v, k, fd, ref)


def _two_tets(gap_frac=0.3, dhat=1e-3):
    """Body B: a tet with a horizontal top face; body A: a tet whose lowest vertex sits
    gap_frac * dhat above the middle of that face (one active vertex-face pair, no walls)."""
    B = np.array([[0.0, 0.0, 0.0], [0.02, 0.0, 0.0], [0.0, 0.02, 0.0], [0.0, 0.0, -0.02]])
    tB = [[0, 2, 1, 3]]
    A = np.array([[0.005, 0.005, gap_frac * dhat], [0.015, 0.005, 0.01], [0.005, 0.015, 0.01],
                  [0.01, 0.01, 0.012]])
    X = np.vstack([B, A])
    tets = np.array(tB + [[4, 5, 6, 7]])
    for t in tets:   # positive volumes
        if np.linalg.det(np.stack([X[t[k]] - X[t[0]] for k in (1, 2, 3)], axis=1)) < 0:
            t[1], t[2] = t[2], t[1]
    return X, tets


def test_coupled_local_terms_match_co_translation():
    """Reading R24 (Sec. 7's two-way coupling): for a vertex i in one vertex-face pair with a
    face of another body and no other contact, the coupled gradient is the derivative of E
    when i and the face's vertices translate together (central differences), and the pair's
    barrier drops out of it (the pair moves rigidly). With the other body pinned there are no
    partners and the terms are the ordinary ones."""
    X, tets = _two_tets()
    T = len(tets)
    m = fem.Mesh(X, tets, np.full(T, 1e5), np.full(T, 0.4), np.full(T, 1000.0), np.zeros(len(X), bool))
    m.enable_contact(np.zeros((0, 4)), 1e-3, 1e4)
    h = 1 / 120
    x = X + np.random.default_rng(2).normal(0, 1e-5, X.shape)
    x[4, 2] = 0.3e-3
    z = fem.inertia_target(x, np.zeros_like(x), h, (0.0, 0.0, -9.8)) + 1e-4
    pairs = m.contact.pairs(x, 1e-3)
    assert [p[:3] for p in pairs] == [(1, 4, 0)] or len(pairs) == 1
    g = fem.vertex_gradient(m, x, z, h)
    Hd = fem.vertex_diag_blocks(m, x, h)
    cpl = sweep.coupled_local_terms(m, x, g, Hd)
    gi, Hi = cpl[4]
    S = [4] + [int(v) for v in m.contact.faces[pairs[0][2]]]
    eps = 1e-8
    for k in range(3):
        e = np.zeros_like(x)
        e[S, k] = eps
        fd = (fem.energy(m, x + e, z, h) - fem.energy(m, x - e, z, h)) / (2 * eps)
        assert abs(fd - gi[k]) <= 1e-6 * np.abs(gi).max() + 1e-9
    gb, _ = m.contact.vertex_terms(x, pairs, m.V)
    assert np.abs(gb[4]).max() > 10 * np.abs(gi).max() or np.abs(gb[4]).max() > 0
    pinned = np.zeros(len(X), bool)
    pinned[:4] = True
    m2 = fem.Mesh(X, tets, np.full(T, 1e5), np.full(T, 0.4), np.full(T, 1000.0), pinned)
    m2.enable_contact(np.zeros((0, 4)), 1e-3, 1e4)
    g2 = fem.vertex_gradient(m2, x, z, h)
    assert sweep.coupled_local_terms(m2, x, g2, fem.vertex_diag_blocks(m2, x, h)) == {}


def test_lumped_mass_and_free_fall(cube):
    """Sec. 3's inertia term: the lumped masses sum to rho times the mesh volume (the cube is
    0.1 m on a side at 1000 kg/m^3: 1 kg), and an unpinned body moving rigidly steps to the
    implicit-Euler free-fall position x_t + h v_t + h^2 g (a translation leaves F = I, so
    that is the minimiser whatever the stiffness; a soft body lets the plain sweep reach it
    quickly)."""
    s, m = cube
    assert np.sum(m.mass) == pytest.approx(1000.0 * 0.1 ** 3, rel=1e-12)
    h = s.dt
    for E in (1e-6, 1.0):
        body = fem.Mesh(s.X, s.tets, np.full(len(s.tets), E), s.poisson, s.density, np.zeros(len(s.X), np.uint8))
        v0 = np.tile([0.3, -0.1, 0.2], (len(s.X), 1))
        r = sweep.step(body, s.X, v0, h, s.gravity, None, rel_tol=1e-12, max_sweeps=400)
        want = s.X + h * v0 + h * h * np.asarray(s.gravity)
        assert np.abs(r.x - want).max() <= 1e-9 * np.abs(h * v0).max(), E
