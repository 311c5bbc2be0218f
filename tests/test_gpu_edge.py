"""GPU edge cases of the step, each against the FP64 oracle: a mesh whose every vertex is
pinned (no DOF: the step is x_{t+1} = x_t after 0 sweeps), a single tet with one free
vertex (no element is remote from it, so every cubature slot is empty), and a zero sweep
cap (the state is returned unchanged with ENOTCONVERGED)."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute, sweep

pytestmark = pytest.mark.gpu


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def single_tet():
    X = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [0.0, 0.01, 0.0], [0.002, 0.003, 0.01]])
    T = np.array([[0, 1, 2, 3]], np.int32)
    pin = np.array([1, 1, 1, 0], np.uint8)
    v0 = np.array([[0.0, 0.0, 0.0]] * 3 + [[0.5, -0.2, 1.0]])
    return scenes.Scene("single tet", X, T, np.array([1e5]), np.array([0.4]), np.array([1000.0]), pin, v0)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_all_pinned_mesh_is_a_converged_zero_sweep_step(cuda, prec):
    s = scenes.cube_scene()
    s.pinned[:] = 1
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 50)
    assert o.converged and o.sweeps == 0
    g = p.Mesh.from_scene(s)
    g.precompute(n_cub=4)
    x, v = t(s.X, cuda), t(np.full_like(s.X, 0.3), cuda)
    rep = g.step(x, v, p.step_opts(precision=prec, max_sweeps=50))
    assert rep.converged == 1 and rep.sweeps == 0 and rep.rel_residual == 0.0
    assert np.array_equal(x.cpu().numpy(), o.x)
    assert np.array_equal(v.cpu().numpy(), np.zeros_like(s.X))
    # the block-size autotuner has nothing to time and keeps the default
    assert g.autotune(x, v, p.step_opts(precision=prec)) in (64, 128, 256)


@pytest.mark.parametrize("prec,tol", [(p.FP64, 1e-9), (p.FP32, 1e-4)])
def test_single_tet_one_free_vertex(cuda, prec, tol):
    s = single_tet()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    cub = precompute.train_cubature(m, s.dt)
    assert np.all(cub.elem < 0)  # the only element touches the only free vertex
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub, 1e-8, 50)
    assert o.converged
    g = p.Mesh.from_scene(s)
    g.precompute_import(cub.elem, cub.weight, cub.ubar)
    x, v = t(s.X, cuda), t(s.v0, cuda)
    rep = g.step(x, v, p.step_opts(precision=prec, max_sweeps=50, rel_tol=1e-8 if prec == p.FP64 else 1e-5))
    xg = x.cpu().numpy()
    if prec == p.FP64:
        assert rep.converged == 1 and rep.sweeps == o.sweeps
    d = o.x - s.X
    assert np.linalg.norm(xg - o.x) <= tol * np.linalg.norm(d)
    assert np.array_equal(xg[:3], s.X[:3])  # pinned corners do not move


def test_zero_sweep_cap_returns_the_state_unchanged(cuda):
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 0)
    assert not o.converged and o.sweeps == 0
    g = p.Mesh.from_scene(s)
    x, v = t(s.X, cuda), t(s.v0, cuda)
    rep = g.step(x, v, p.step_opts(precision=p.FP64, correction=p.CORR_OFF, max_sweeps=0))
    assert rep.converged == 0 and rep.sweeps == 0 and abs(rep.rel_residual - 1.0) < 1e-12
    assert np.array_equal(x.cpu().numpy(), s.X)
    assert np.array_equal(v.cpu().numpy(), np.zeros_like(s.X))


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_non_finite_state_is_reported_and_left_alone(cuda, prec):
    """A NaN position makes the first residual non-finite: the step stops with
    JGS2_EDIVERGED and writes nothing back."""
    s = scenes.cube_scene()
    g = p.Mesh.from_scene(s)
    x0 = s.X.copy()
    x0[3] = np.nan  # a free vertex
    x, v = t(x0, cuda), t(s.v0, cuda)
    with pytest.raises(p.JGS2Error) as err:
        g.step(x, v, p.step_opts(precision=prec, correction=p.CORR_OFF, max_sweeps=10))
    assert err.value.status == 6
    xa = x.cpu().numpy()
    assert np.all(np.isnan(xa[3])) and np.array_equal(np.delete(xa, 3, axis=0), np.delete(x0, 3, axis=0))
    assert np.array_equal(v.cpu().numpy(), s.v0)
