"""Pins of the oracle's Gauss-Seidel mode (Sec. 8.1, oracle/gs.py) on the 384-tet cube:
the colouring is valid and greedy; the generalised sub-problem's U_bar satisfies its
constraints and equilibrium, and reduces to the Jacobi U_bar (Eq. u) when every group is
a single vertex, as does its cubature training; with every vertex in one group a GS sweep
is the Jacobi sweep; the projected-Newton minimiser is a fixed point of the GS sweep."""
import numpy as np
import pytest

import scenes
from oracle import fem, gs, newton, precompute, sweep


@pytest.fixture(scope="module")
def cube():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return s, m


def test_colouring_is_valid_and_greedy(cube):
    s, m = cube
    col = gs.greedy_colouring(m)
    assert np.all(col[m.pinned] == -1) and np.all(col[m.free] >= 0)
    nbr = [set() for _ in range(m.V)]
    for t in m.tets:
        for a in t:
            nbr[a].update(int(b) for b in t if b != a)
    for v in m.free:
        assert all(col[u] != col[v] for u in nbr[v] if not m.pinned[u])   # valid
        earlier = {col[u] for u in nbr[v] if u < v and not m.pinned[u]}
        assert col[v] == min(set(range(len(earlier) + 1)) - earlier)      # greedy, caller order
    assert col.max() + 1 <= 15   # at most (max degree + 1) colours


def test_group_ubar_constraints_and_equilibrium(cube):
    s, m = cube
    Hbar = precompute.rest_hessian(m, s.dt)
    col = gs.greedy_colouring(m)
    Ub = gs.ubar_groups(m, Hbar, col)
    fcol = col[m.free]
    for d in range(0, m.free.size, 7):
        G = np.nonzero(fcol == fcol[d])[0]
        gd = (3 * G[:, None] + np.arange(3)).ravel()
        C = np.setdiff1d(np.arange(Hbar.shape[0]), gd)
        assert np.allclose(Ub[d][3 * d:3 * d + 3], np.eye(3))
        others = [g for g in G if g != d]
        for o in others:
            assert np.all(Ub[d][3 * o:3 * o + 3] == 0.0)
        # unconstrained DOFs in equilibrium: rows C of H_bar U_bar vanish (Eq. cms)
        assert np.max(np.abs((Hbar @ Ub[d])[C])) <= 1e-9 * np.max(np.abs(Hbar))


def test_single_vertex_groups_reduce_to_jacobi(cube):
    s, m = cube
    Hbar = precompute.rest_hessian(m, s.dt)
    single = -np.ones(m.V, dtype=np.int64)
    single[m.free] = np.arange(m.free.size)
    Ub_g = gs.ubar_groups(m, Hbar, single)
    Ub_j, _ = precompute.ubar_all(m, Hbar)
    assert np.max(np.abs(Ub_g - Ub_j)) <= 1e-10 * np.max(np.abs(Ub_j))
    cg = gs.train_cubature_gs(m, s.dt, single, Hbar=Hbar)
    cj = precompute.train_cubature(m, s.dt, Hbar=Hbar)
    assert np.array_equal(cg.elem, cj.elem)
    assert np.allclose(cg.weight, cj.weight, rtol=1e-7, atol=1e-10)


def test_one_group_sweep_is_the_jacobi_sweep(cube):
    s, m = cube
    cub = precompute.train_cubature(m, s.dt)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    x = scenes.perturbed_state(s.X, s.pinned, 2e-3, seed=4)
    one = np.where(m.pinned, -1, 0)
    assert np.array_equal(gs.gs_sweep(m, x, z, s.dt, one, cub), sweep.run_sweeps(m, x, z, s.dt, cub, 1))


def test_newton_minimiser_is_a_gs_fixed_point(cube):
    s, m = cube
    col = gs.greedy_colouring(m)
    cub = gs.train_cubature_gs(m, s.dt, col)
    xs, _, _ = newton.newton_solve(m, s.X, s.v0, s.dt, s.gravity, rel_tol=1e-12)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    x1 = gs.gs_sweep(m, xs, z, s.dt, col, cub)
    assert np.linalg.norm(x1 - xs) <= 1e-9 * np.linalg.norm(xs - s.X)


def test_gs_beats_jacobi_without_correction(cube):
    """Plain nonlinear GS (no correction) against plain Jacobi, both with the line search:
    fewer sweeps to 1e-4 (a claim check, not parity)."""
    s, m = cube
    col = gs.greedy_colouring(m)
    o_gs = gs.gs_step(m, s.X, s.v0, s.dt, s.gravity, col, None, rel_tol=1e-4, max_sweeps=400)
    o_j = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 400)
    assert o_gs.converged and o_j.converged and o_gs.sweeps < o_j.sweeps
