"""GPU parity of the cloth path (jgs2_cloth_*, reading R26) against the oracle's cloth
(oracle/cloth.py, pinned in tests/test_oracle_cloth.py): energy and gradient (FP64 1e-10),
sweeps (FP64 1e-9, FP32 1e-4 per vertex), a whole FP64 step (sweep count, positions), and a
step that converges."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import cloth

pytestmark = pytest.mark.gpu

TOL = {p.FP64: 1e-9, p.FP32: 1e-4}


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def ocloth(s):
    return cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned)


def state(s, seed, scale=0.01):
    r = np.random.default_rng(seed)
    x = s.X + r.normal(0.0, scale, s.X.shape)
    x[s.pinned.astype(bool)] = s.X[s.pinned.astype(bool)]
    return x


@pytest.mark.parametrize("n", [5, 21])
def test_cloth_energy_gradient(cuda, n):
    s = scenes.cloth_scene(n=n, vel_sigma=0.05)
    o = ocloth(s)
    x = state(s, 1)
    z = cloth.inertia_target(s.X, s.v0, s.dt, s.gravity)
    c = p.Cloth.from_scene(s)
    E, g = c.energy_gradient(t(s.X, cuda), t(s.v0, cuda), t(x, cuda))
    go = o.gradient(x, z, s.dt)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-10 * np.abs(go).max()
    assert abs(E - o.energy(x, z, s.dt)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
@pytest.mark.parametrize("ls", [1, 0])
def test_cloth_sweeps(cuda, prec, ls):
    s = scenes.cloth_scene(n=21, vel_sigma=0.05)
    o = ocloth(s)
    x = state(s, 2, 0.002)
    z = cloth.inertia_target(s.X, s.v0, s.dt, s.gravity)
    c = p.Cloth.from_scene(s)
    xg = t(x, cuda)
    c.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 3, p.step_opts(precision=prec, line_search=ls))
    xo = cloth.run_sweeps(o, x, z, s.dt, 3, line_search_on=bool(ls))
    disp = np.linalg.norm(xo - x, axis=1).max()
    err = np.linalg.norm(xg.cpu().numpy() - xo, axis=1).max() / disp
    assert err <= TOL[prec], err


def test_cloth_step_fp64_matches_oracle(cuda):
    s = scenes.cloth_scene(n=11)
    o = ocloth(s)
    c = p.Cloth.from_scene(s)
    x, v = t(s.X, cuda), t(s.v0, cuda)
    rep = c.step(x, v, p.step_opts(precision=p.FP64, max_sweeps=60, rel_tol=1e-4, check_every=7))
    r = cloth.step(o, s.X, s.v0, s.dt, s.gravity, rel_tol=1e-4, max_sweeps=60)
    assert rep.sweeps == r.sweeps
    assert bool(rep.converged) == r.converged
    assert np.linalg.norm(x.cpu().numpy() - r.x) / np.linalg.norm(r.x - s.X) <= 1e-9
    assert np.abs(v.cpu().numpy() - r.v).max() <= 1e-6 * np.abs(r.v).max()


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_cloth_step_converges(cuda, prec):
    s = scenes.cloth_scene(n=11, youngs=1e5)
    c = p.Cloth.from_scene(s)
    x, v = t(s.X, cuda), t(s.v0, cuda)
    rep = c.step(x, v, p.step_opts(precision=prec, max_sweeps=5000, rel_tol=1e-4))
    assert rep.converged and rep.rel_residual <= 1e-4
    # the cloth fell (gravity) and the pins held
    xs = x.cpu().numpy()
    pin = s.pinned.astype(bool)
    assert np.all(xs[~pin, 2] < 0.0)
    assert np.abs(xs[pin] - s.X[pin]).max() == 0.0


def ocloth_walls(s):
    return cloth.Cloth(s.X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned,
                       planes=s.planes, dhat=s.dhat, kappa=s.kappa)


def test_cloth_walls_energy_gradient(cuda):
    s = scenes.cloth_floor_scene()
    o = ocloth_walls(s)
    x = s.X + np.random.default_rng(3).normal(0.0, 1e-4, s.X.shape)
    d = o.wall_distances(x)
    assert np.all((d > 0) & (d < s.dhat))
    z = cloth.inertia_target(s.X, s.v0, s.dt, s.gravity)
    c = p.Cloth.from_scene(s)
    E, g = c.energy_gradient(t(s.X, cuda), t(s.v0, cuda), t(x, cuda))
    go = o.gradient(x, z, s.dt)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-10 * np.abs(go).max()
    assert abs(E - o.energy(x, z, s.dt)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_cloth_walls_sweeps_and_step(cuda, prec):
    s = scenes.cloth_floor_scene()
    o = ocloth_walls(s)
    c = p.Cloth.from_scene(s)
    x = s.X + np.random.default_rng(4).normal(0.0, 1e-4, s.X.shape)
    z = cloth.inertia_target(s.X, s.v0, s.dt, s.gravity)
    xg = t(x, cuda)
    c.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 3, p.step_opts(precision=prec))
    xo = cloth.run_sweeps(o, x, z, s.dt, 3)
    disp = np.linalg.norm(xo - x, axis=1).max()
    assert np.linalg.norm(xg.cpu().numpy() - xo, axis=1).max() / disp <= TOL[prec]
    # a whole step: above the floor, and (FP64) the oracle's sweep count and positions
    xs, vs = t(s.X, cuda), t(s.v0, cuda)
    rep = c.step(xs, vs, p.step_opts(precision=prec, max_sweeps=400, rel_tol=1e-4))
    assert xs.cpu().numpy()[:, 2].min() > 0.0
    if prec == p.FP64:
        r = cloth.step(o, s.X, s.v0, s.dt, s.gravity, rel_tol=1e-4, max_sweeps=400)
        assert rep.sweeps == r.sweeps
        assert np.linalg.norm(xs.cpu().numpy() - r.x) / np.linalg.norm(r.x - s.X) <= 1e-9
