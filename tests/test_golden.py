"""The oracle against its stored values (tests/golden/, written by make_golden.py from
oracle/ only): the cube's greedy cubature sets (Sec. 5) and one implicit-Euler step
(Sec. 3) by JGS2 and by uncorrected Jacobi sweeps. A change to the oracle's arithmetic
that moves these values fails here until the fixtures are regenerated with it."""
import importlib.util
import os

import numpy as np
import pytest

import scenes
from oracle import fem, precompute, sweep

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)


@pytest.fixture(scope="module")
def cube():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return s, m, precompute.train_cubature(m, s.dt)


def test_cubature_sets_match_golden(cube):
    _, _, cub = cube
    elem, w = golden.load_cubature(os.path.join(HERE, "cube_cubature.txt"))
    assert np.array_equal(cub.elem, elem)
    assert np.allclose(cub.weight, w, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("name,corrected", [("cube_jgs2_step.txt", True), ("cube_jacobi_step.txt", False)])
def test_step_matches_golden(cube, name, corrected):
    s, m, cub = cube
    sweeps, conv, res, x = golden.load_step(os.path.join(HERE, name))
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub if corrected else None, golden.REL_TOL, golden.MAX_SWEEPS)
    assert o.sweeps == sweeps and o.converged == conv
    assert np.allclose(o.residuals, res, rtol=1e-9, atol=1e-14)
    assert np.linalg.norm(o.x - x) <= 1e-12 * np.linalg.norm(x - s.X)
