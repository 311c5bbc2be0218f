"""Pins of the oracle's lagged wall friction (reading R25: IPC's friction potential on the
vertex-wall pairs, lagged normal forces from the step start) to what fixes it independently
of its own code:
- the smoothing f0 and its derivative (closed forms and continuity at the slip eps);
- finite differences of the friction energy's gradient and of the diagonal blocks;
- momentum balance of a converged step: the walls' barrier pushes along the wall normal and
  internal elastic forces cancel in sum, so the block's tangential momentum changes by the
  friction impulse alone. Sliding (every contact vertex slips by more than eps) that impulse
  is -h mu sum_v lam_v u_v/|u_v|, Coulomb's law with the lagged normal forces; sticking it is
  at most h mu sum lam_v in norm.
"""
import numpy as np
import pytest

import scenes
from oracle import contact, fem


def test_f0_closed_forms():
    eps = 2e-4
    assert contact.friction_f0(0.0, eps) == pytest.approx(eps / 3.0, rel=1e-15)
    # C^1 at eps: value eps and slope 1 from both sides
    lo, hi = eps * (1 - 1e-9), eps * (1 + 1e-9)
    assert contact.friction_f0(lo, eps) == pytest.approx(eps, rel=1e-8)
    assert contact.friction_f0(hi, eps) == pytest.approx(eps, rel=1e-8)
    assert contact.friction_f1(lo, eps) == pytest.approx(1.0, rel=1e-8)
    for y in (0.1 * eps, 0.5 * eps, 0.9 * eps, 2 * eps, 10 * eps):
        fd = (contact.friction_f0(y + 1e-12, eps) - contact.friction_f0(y - 1e-12, eps)) / 2e-12
        assert contact.friction_f1(y, eps) == pytest.approx(float(fd), rel=1e-5)
        assert contact.friction_f1_over_y(y, eps) == pytest.approx(float(contact.friction_f1(y, eps)) / y,
                                                                   rel=1e-13)
    assert contact.friction_f1_over_y(0.0, eps) == pytest.approx(2.0 / eps)


def block_on_floor(mu=0.5, speed=0.0, nv=3, size=0.02, gap=9.8e-4, E=1e7, kappa=1e4):
    """A small stiff block just above the floor (z >= 0), moving along it. The gap (0.98 dhat)
    puts the barrier force near the block's weight, so the lagged normal forces are those of a
    block at rest on the floor."""
    X, tets = scenes.kuhn_grid(nv, nv, nv, (size, size, size))
    X = X + np.array([0.0, 0.0, gap])
    T = len(tets)
    m = fem.Mesh(X, tets, np.full(T, E), np.full(T, 0.4), np.full(T, 1000.0), np.zeros(len(X), np.uint8))
    m.enable_contact(np.array([[0.0, 0.0, 1.0, 0.0]]), 1e-3, kappa, friction_mu=mu, friction_eps_v=1e-3)
    v0 = np.zeros_like(X)
    v0[:, 0] = speed
    v0[:, 1] = 0.4 * speed
    return m, X, v0


def test_friction_gradient_and_blocks_by_finite_differences():
    m, X, v0 = block_on_floor(mu=0.4)
    h = 1.0 / 100
    m.contact.lag_friction(X, h)
    rng = np.random.default_rng(3)
    eps = 1e-3 * h
    for scale in (0.3 * eps, 3 * eps):  # both branches of f0
        x = X + rng.normal(size=X.shape) * scale
        g, H = m.contact.friction_terms(x, m.V)
        lam = m.contact.fr[1][:, 0]
        assert np.count_nonzero(lam) > 0
        for v in np.nonzero(lam)[0][:4]:
            for a in range(3):
                e = np.zeros_like(x)
                e[v, a] = 1e-7 * scale
                fd = (m.contact.friction_energy(x + e) - m.contact.friction_energy(x - e)) / (2 * e[v, a])
                assert g[v, a] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())
                g1, _ = m.contact.friction_terms(x + e, m.V)
                g0, _ = m.contact.friction_terms(x - e, m.V)
                fdH = (g1[v] - g0[v]) / (2 * e[v, a])
                assert np.allclose(H[v][:, a], fdH, rtol=1e-4, atol=1e-6 * np.abs(H[v]).max())
            # positive semidefinite on both branches
            assert np.linalg.eigvalsh(H[v]).min() >= -1e-9 * np.abs(H[v]).max()


def newton_step(m, X, v0, h, grav):
    """Converged implicit-Euler step of the block (dense Newton on the free DOFs, Armijo on
    the total energy): elastic and inertial Hessian plus the vertex-diagonal barrier and
    friction blocks (exact for a floor-only scene: every contact term is per vertex)."""
    z = fem.inertia_target(X, v0, h, grav)
    m.contact.lag_friction(X, h)
    x = X.copy()
    g0 = None
    for _ in range(60):
        g = fem.vertex_gradient(m, x, z, h)
        gn = np.linalg.norm(g)
        g0 = gn if g0 is None else g0
        if gn <= 1e-9 * g0:
            break
        H = fem.global_hessian(m, x, h, psd=True)
        pairs = m.contact.pairs(x, m.contact.dhat)
        _, Hb = m.contact.vertex_terms(x, pairs, m.V)
        _, Hf = m.contact.friction_terms(x, m.V)
        for v in range(m.V):
            H[3 * v:3 * v + 3, 3 * v:3 * v + 3] += Hb[v] + Hf[v]
        d = np.linalg.solve(H, -g.reshape(-1)).reshape(-1, 3)
        # stay inside the barrier's domain, then Armijo on E
        a = 1.0
        while np.any(x[:, 2] + a * d[:, 2] <= 0.1 * np.min(x[:, 2])):
            a *= 0.5
        e0 = fem.energy(m, x, z, h)
        slope = float(np.sum(g * d))
        while fem.energy(m, x + a * d, z, h) > e0 + 1e-4 * a * slope and a > 1e-6:
            a *= 0.5
        if a <= 1e-6:
            # below the energy's rounding: Newton's full step, if it lowers |g|
            if np.linalg.norm(fem.vertex_gradient(m, x + d, z, h)) >= gn:
                break
            a = 1.0
        x = x + a * d
    res = np.linalg.norm(fem.vertex_gradient(m, x, z, h))
    assert res <= 1e-8 * g0
    return x, res


def test_sliding_block_loses_the_coulomb_impulse():
    h = 1.0 / 100
    grav = (0.0, 0.0, -9.8)
    m, X, v0 = block_on_floor(mu=0.3, speed=0.5)
    x, res = newton_step(m, X, v0, h, grav)
    _, lam, eps = m.contact.fr
    lam = lam[:, 0]
    slip = (x - X)[:, :2]
    on = lam > 0
    assert on.sum() >= 4
    assert np.all(np.linalg.norm(slip[on], axis=1) > eps)  # every contact vertex slides
    dp = np.sum(m.mass[:, None] * ((x - X) / h - v0)[:, :2], axis=0)
    coulomb = -h * m.contact.mu * np.sum(lam[on, None] * slip[on] / np.linalg.norm(slip[on], axis=1)[:, None],
                                         axis=0)
    # equal up to the solve's residual force (the sum of the gradient's tangential rows)
    assert np.linalg.norm(dp - coulomb) <= 1e-6 * np.linalg.norm(coulomb) + h * np.sqrt(m.V) * res
    # and the impulse opposes the motion
    assert float(dp @ v0[0, :2]) < 0


def test_sticking_block_stays_within_the_friction_cone():
    h = 1.0 / 100
    grav = (0.0, 0.0, -9.8)
    m, X, v0 = block_on_floor(mu=0.8, speed=2e-4)
    x, res = newton_step(m, X, v0, h, grav)
    _, lam, eps = m.contact.fr
    lam = lam[:, 0]
    on = lam > 0
    slip = np.linalg.norm((x - X)[on, :2], axis=1)
    assert np.all(slip < eps)  # static branch
    dp = np.sum(m.mass[:, None] * ((x - X) / h - v0)[:, :2], axis=0)
    assert np.linalg.norm(dp) <= h * m.contact.mu * lam.sum() * (1 + 1e-9) + h * np.sqrt(m.V) * res
    # the tangential motion was nearly stopped: the block keeps well under its initial slip
    assert slip.max() < 0.5 * 2e-4 * h * np.hypot(1.0, 0.4)
