"""Pins of the oracle's cloth (reading R26: StVK membrane triangles, quadratic bending on
interior edges, the per-vertex Jacobi sweep with the global line search) to what fixes it
independently of its own code: the StVK energy of a uniaxial stretch in closed form; zero
membrane energy under rigid motions; the bending weights' defining properties (they sum
to zero and annihilate a flat rest hinge, so affine images of a flat sheet cost nothing);
the bending energy of a cylinder scaling as the squared curvature; finite differences of
the gradient and of the diagonal blocks; and the sweep's fixed point against a Newton
solve of the same step."""
import numpy as np
import pytest

import scenes
from oracle import cloth


def single(Y=1e6, nu=0.3, t=1e-3, rho=200.0, bend=0.0):
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    return cloth.Cloth(X, np.array([[0, 1, 2]]), Y, nu, t, rho, bend)


def test_uniaxial_stretch_closed_form():
    Y, nu, t = 2e6, 0.3, 1e-3
    c = single(Y, nu, t)
    mu, lam = Y * t / (2 * (1 + nu)), Y * t * nu / (1 - nu * nu)
    for s in (0.7, 1.0, 1.2, 2.0):
        x = c.X * np.array([s, 1.0, 1.0])
        e = 0.5 * (s * s - 1.0)
        ref = 0.5 * (mu * e * e + 0.5 * lam * e * e)  # area 1/2
        em, _, _, _ = c.membrane(x)
        assert em[0] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_membrane_rigid_motion_invariance():
    s = scenes.cloth_scene(n=6)
    c = cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, 0.0)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(1.1), -np.sin(1.1)], [0, np.sin(1.1), np.cos(1.1)]])
    x = s.X @ R.T + np.array([0.3, -0.2, 1.0])
    em, _, _, _ = c.membrane(x)
    assert np.abs(em).max() <= 1e-20
    assert np.sum(c.membrane(s.X * 1.1)[0]) > 0


def test_bending_weights_annihilate_flat_hinges():
    r = np.random.default_rng(0)
    for _ in range(20):
        P = np.hstack([r.uniform(-1, 1, (4, 2)), np.zeros((4, 1))])
        # a convex quad split along (0, 1): vertices 2 and 3 on either side
        P[0], P[1] = [-1.0, 0.0, 0.0], [1.0, 0.0, 0.0]
        P[2, 1], P[3, 1] = abs(P[2, 1]) + 0.1, -abs(P[3, 1]) - 0.1
        A = r.normal(size=(3, 3))
        X = P @ A.T  # an arbitrary plane in space
        c = cloth.Cloth(X, np.array([[0, 1, 2], [1, 0, 3]]), 1e6, 0.3, 1e-3, 200.0, 1.0)
        assert len(c.hinges) == 1
        K = c.K[0]
        assert abs(K.sum()) <= 1e-12 * np.abs(K).max()
        assert np.abs(K @ X[c.hinges[0]]).max() <= 1e-12 * np.abs(K).max() * np.abs(X).max()


def test_affine_images_of_a_flat_sheet_have_no_bending_energy():
    s = scenes.cloth_scene(n=7)
    c = cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, 1e-3)
    A = np.random.default_rng(1).normal(size=(3, 3))
    w = c.bending_w(s.X @ A.T + 0.3)
    assert np.abs(w).max() <= 1e-12
    # and a bent sheet does
    x = s.X.copy()
    x[:, 2] = 0.1 * np.sin(3 * x[:, 0])
    assert np.abs(c.bending_w(x)).max() > 1e-3


def test_cylinder_bending_scales_with_squared_curvature():
    s = scenes.cloth_scene(n=41, size=0.2)
    c = cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, 1.0)

    def roll(R):  # isometric: wrap the x axis onto a cylinder of radius R
        x = s.X.copy()
        x[:, 0] = R * np.sin(s.X[:, 0] / R)
        x[:, 2] = R * (1 - np.cos(s.X[:, 0] / R))
        return x

    e = []
    for R in (0.4, 0.8):
        w = c.bending_w(roll(R))
        e.append(0.5 * np.sum(c.kb * np.sum(w * w, 1)))
    assert e[0] / e[1] == pytest.approx(4.0, rel=1e-2)


def test_gradient_and_blocks_by_finite_differences():
    s = scenes.cloth_scene(n=5)
    c = cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, 1e-3, s.pinned)
    r = np.random.default_rng(2)
    x = s.X + r.normal(0.0, 0.01, s.X.shape)
    x[c.pinned] = s.X[c.pinned]
    h = s.dt
    z = cloth.inertia_target(s.X, s.v0, h, s.gravity)
    g = c.gradient(x, z, h)
    H = c.diag_blocks(x, h, project=False)
    for v in c.free[:8]:
        for a in range(3):
            e = np.zeros_like(x)
            e[v, a] = 1e-6
            fd = (c.energy(x + e, z, h) - c.energy(x - e, z, h)) / 2e-6
            assert g[v, a] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g).max())
            fdH = (c.gradient(x + e, z, h)[v] - c.gradient(x - e, z, h)[v]) / 2e-6
            assert np.allclose(H[v][:, a], fdH, rtol=1e-5, atol=1e-8 * np.abs(H[v]).max())
    Hp = c.diag_blocks(x, h)
    assert np.all(np.linalg.eigvalsh(Hp[c.free]) > 0)


def test_sweeps_reach_the_newton_solution():
    s = scenes.cloth_scene(n=5, youngs=1e5)
    c = cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned)
    h = s.dt
    z = cloth.inertia_target(s.X, s.v0, h, s.gravity)
    # Newton on the free DOFs with a finite-difference Hessian of the gradient
    x = s.X.copy()
    fr = c.free
    for _ in range(30):
        g = c.gradient(x, z, h)[fr].ravel()
        if np.linalg.norm(g) < 1e-12:
            break
        n = g.size
        Hn = np.zeros((n, n))
        for k in range(n):
            e = np.zeros_like(x)
            e[fr[k // 3], k % 3] = 1e-7
            Hn[:, k] = (c.gradient(x + e, z, h)[fr].ravel() - c.gradient(x - e, z, h)[fr].ravel()) / 2e-7
        d = np.linalg.solve(0.5 * (Hn + Hn.T), -g).reshape(-1, 3)
        a = 1.0
        e0 = c.energy(x, z, h)
        while True:
            xn = x.copy()
            xn[fr] += a * d
            if c.energy(xn, z, h) <= e0 + 1e-4 * a * float(g @ d.ravel()) or a < 1e-8:
                break
            a *= 0.5
        x = xn
    assert np.linalg.norm(c.gradient(x, z, h)[fr]) < 1e-9
    r = cloth.step(c, s.X, s.v0, h, s.gravity, rel_tol=1e-8, max_sweeps=5000)
    assert r.converged
    assert np.abs(r.x - x).max() <= 1e-5 * np.abs(x - s.X).max()


def floor_cloth(n=5, gap=6e-4):
    s = scenes.cloth_scene(n=n, youngs=1e5)
    X = s.X + np.array([0.0, 0.0, gap])
    c = cloth.Cloth(X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned,
                    planes=np.array([[0.0, 0.0, 1.0, 0.0]]), dhat=1e-3, kappa=1e2)
    return s, X, c


def test_wall_barrier_by_finite_differences():
    s, X, c = floor_cloth()
    r = np.random.default_rng(5)
    x = X + r.normal(0.0, 1e-4, X.shape)
    x[c.pinned] = X[c.pinned]
    h = s.dt
    z = cloth.inertia_target(X, s.v0, h, s.gravity)
    g = c.gradient(x, z, h)
    H = c.diag_blocks(x, h, project=False)
    d = c.wall_distances(x)
    assert np.all((d > 0) & (d < c.dhat))  # every free vertex feels the barrier
    for v in c.free[:6]:
        for a in range(3):
            e = np.zeros_like(x)
            e[v, a] = 1e-9
            fd = (c.energy(x + e, z, h) - c.energy(x - e, z, h)) / 2e-9
            assert g[v, a] == pytest.approx(fd, rel=1e-5, abs=1e-8 * np.abs(g).max())
    # the barrier's block is its Gauss-Newton (here exact) second derivative along n
    Hn = c.diag_blocks(x, h, project=False)
    c0 = cloth.Cloth(X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned)
    Hw = Hn - c0.diag_blocks(x, h, project=False)
    v = c.free[0]
    fd = (c.gradient(x + np.eye(3)[2] * 1e-9 * (np.arange(len(x)) == v)[:, None], z, h)[v, 2] -
          c0.gradient(x + np.eye(3)[2] * 1e-9 * (np.arange(len(x)) == v)[:, None], z, h)[v, 2] -
          (c.gradient(x, z, h)[v, 2] - c0.gradient(x, z, h)[v, 2])) / 1e-9
    assert Hw[v][2, 2] == pytest.approx(fd, rel=1e-4)
    assert abs(Hw[v][0, 0]) + abs(Hw[v][0, 2]) <= 1e-12 * abs(Hw[v][2, 2])


def test_cloth_on_the_floor_stays_above_it_and_converges():
    s, X, c = floor_cloth()
    h = s.dt
    r = cloth.step(c, X, s.v0, h, s.gravity, rel_tol=1e-6, max_sweeps=20000)
    assert r.converged
    d = c.wall_distances(r.x)
    assert d.min() > 0.0
    # at the converged state the barrier holds the sheet up: it sank, but less than a free
    # fall would take it
    c0 = cloth.Cloth(X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned)
    r0 = cloth.step(c0, X, s.v0, h, s.gravity, rel_tol=1e-6, max_sweeps=20000)
    free = c.free
    assert np.all(r.x[free, 2] >= r0.x[free, 2] - 1e-12)
    assert np.any(r.x[free, 2] > r0.x[free, 2] + 1e-9)


def test_lumped_mass_and_free_fall():
    """The cloth's lumped masses sum to rho t times its area (a 0.5 m square, 200 kg/m^3,
    5e-4 m thick: 0.025 kg), and an unpinned cloth moving rigidly steps to the
    implicit-Euler free-fall position x_t + h v_t + h^2 g (a translation changes neither
    the membrane strain nor the bending vectors)."""
    s = scenes.cloth_scene(n=6)
    c = cloth.Cloth(s.X, s.tris, 1e-3, s.poisson, s.thickness, s.density, 1e-9)
    assert np.sum(c.mass) == pytest.approx(s.density * s.thickness * 0.5 ** 2, rel=1e-12)
    assert np.sum(c.area) == pytest.approx(0.5 ** 2, rel=1e-12)
    h = s.dt
    v0 = np.tile([0.2, 0.1, -0.3], (len(s.X), 1))
    r = cloth.step(c, s.X, v0, h, s.gravity, rel_tol=1e-12, max_sweeps=400)
    want = s.X + h * v0 + h * h * np.asarray(s.gravity)
    assert np.abs(r.x - want).max() <= 1e-9 * np.abs(h * v0).max()
