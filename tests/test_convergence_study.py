"""Findings of the convergence study (tests/convergence_study.py) on the 384-tet cube,
asserted so that a change to the oracle's correction that moves them is noticed.

  * Sec. 4.2's theorem holds for the exact subspace: with the Schur-complement local
    matrix and the full complement sum of the reduced gradient, one sweep at the rest state
    is the Newton step (iteration operator zero).
  * The cubature-sampled assembled-gradient reading (asm, any training set tried) has an
    iteration operator of spectral radius above 1, and no fixed damping factor brings it
    below 1 (the preconditioned operator has eigenvalues with negative real part): without
    a global safeguard the plain sweep diverges. The element-gradient reading (elem) also
    overshoots undamped but converges with a fixed damping factor, to a biased point.
  * The cubature Hessian alone (no gradient term) is a damped Jacobi iteration.
  * With the global line search (reading R17) the corrected sweep reaches 1e-4 on the cube
    in at most 100x projected Newton's iterations, and in fewer sweeps than uncorrected
    Jacobi; the paper reports 1.1-1.5x Newton (Sec. 8.2-8.3), which no reading here reaches.
"""
import numpy as np
import pytest

import convergence_study as cs
from oracle import precompute, sweep


@pytest.fixture(scope="module")
def cube_ops():
    s = cs.cube()
    m = cs.mesh_of(s)
    H = precompute.rest_hessian(m, s.dt)
    cubs = {nt: precompute.train_cubature(m, s.dt, n_train=nt, Hbar=H) for nt in (4, 20)}
    ops = {nt: cs.linear_operators(m, s.dt, c, H) for nt, c in cubs.items()}
    return s, m, cubs, ops


def test_exact_subspace_sweep_is_the_newton_step(cube_ops):
    _, _, _, ops = cube_ops
    rho, _, _ = cs.spectral_summary(ops[20], "schur", "exact")
    assert rho < 1e-8


@pytest.mark.parametrize("nt", [4, 20])
def test_assembled_gradient_reading_needs_a_global_safeguard(cube_ops, nt):
    _, _, _, ops = cube_ops
    rho, min_re, best = cs.spectral_summary(ops[nt], "cub", "asm")
    assert rho > 1.0 and best > 1.0
    assert min_re < 0.0   # a direction that increases the energy for some modes


@pytest.mark.parametrize("nt", [4, 20])
def test_element_gradient_reading_is_a_damped_iteration(cube_ops, nt):
    """The literal element-gradient term acts on the displacement from rest, not on the
    residual: the plain sweep still overshoots (rho > 1), a fixed damping factor makes it
    converge, and its fixed point is not the minimiser (reading R3)."""
    _, _, _, ops = cube_ops
    rho, min_re, best = cs.spectral_summary(ops[nt], "cub", "elem")
    assert rho > 1.0 and best < 1.0 and min_re > 0.0


def test_cubature_hessian_alone_is_damped_jacobi(cube_ops):
    _, _, _, ops = cube_ops
    rho_j, _, best_j = cs.spectral_summary(ops[20], "jacobi", "none")
    rho_d, min_re, best_d = cs.spectral_summary(ops[20], "cub", "none")
    assert min_re > 0.0                    # positive definite preconditioner: descent directions
    assert rho_d <= rho_j                  # the damper shrinks the largest overshoot
    assert best_d < 1.0 and best_j < 1.0   # both converge once damped
    assert abs(best_d - best_j) < 0.01     # ... at the same first-order rate


def test_globalised_sweeps_against_projected_newton(cube_ops):
    s, m, cubs, _ = cube_ops
    n_newton = cs.newton_iterations(s)
    a = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cubs[20], 1e-4, 1000)
    b = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 1000)
    assert a.converged and b.converged
    assert a.sweeps <= 100 * n_newton
    assert a.sweeps < b.sweeps
