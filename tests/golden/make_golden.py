#!/usr/bin/env python
"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone
(oracle/ for the arithmetic, scenes/ for the seeded inputs). Nothing here reads the CUDA
library. Run from the repository root:

    python tests/golden/make_golden.py

The paper prints no worked example with numbers, so these fixtures are regression values
of the oracle on the 384-tet cube (5x5x5 Kuhn grid, 0.1 m, top face pinned, E = 1e5,
nu = 0.4, rho = 1000, h = 1/120, at rest, gravity (0, 0, -9.8)):

  cube_cubature.txt     the greedy NNLS cubature sets (Sec. 5, Eq. cubature_weight),
                        element ids and weights per free vertex, seed 0
  cube_jgs2_step.txt    one implicit-Euler step (Sec. 3) by JGS2 sweeps with that
                        cubature (asm correction, Armijo line search): r_k per sweep and
                        x_{t+1}
  cube_jacobi_step.txt  the same step with the uncorrected per-vertex Newton sweep

A change to the oracle's arithmetic that moves these values regenerates them in the same
commit, whose message names the passage of the paper (or the reading of it) behind it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402
from oracle import fem, precompute, sweep  # noqa: E402

REL_TOL = 1e-4
MAX_SWEEPS = 400


def cube():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return s, m


def write_step(path, title, res):
    with open(path, "w") as f:
        f.write(f"# {title}\n")
        f.write(f"# rel_tol {REL_TOL:g}, max_sweeps {MAX_SWEEPS}; written by make_golden.py from oracle/\n")
        f.write(f"sweeps {res.sweeps}\nconverged {int(res.converged)}\n")
        f.write(f"residuals {len(res.residuals)}\n")
        for r in res.residuals:
            f.write(f"{r:.17e}\n")
        f.write(f"x {len(res.x)}\n")
        for row in res.x:
            f.write(" ".join(f"{q:.17e}" for q in row) + "\n")


def load_step(path):
    """(sweeps, converged, residuals [n], x [V,3]) from a step fixture."""
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    sweeps, conv, nr = int(rows[0][1]), bool(int(rows[1][1])), int(rows[2][1])
    res = np.array([float(r[0]) for r in rows[3:3 + nr]])
    nx = int(rows[3 + nr][1])
    x = np.array([[float(q) for q in r] for r in rows[4 + nr:4 + nr + nx]])
    return sweeps, conv, res, x


def load_cubature(path):
    """(elem [V,4] int, weight [V,4]) from the cubature fixture."""
    a = np.loadtxt(path, comments="#")
    return a[:, :4].astype(np.int64), a[:, 4:]


def main():
    s, m = cube()
    cub = precompute.train_cubature(m, s.dt)
    with open(os.path.join(HERE, "cube_cubature.txt"), "w") as f:
        f.write("# greedy NNLS cubature sets (Sec. 5, Eq. cubature_weight) of the 384-tet cube, seed 0\n")
        f.write("# per vertex (caller order; pinned vertices and empty slots -1 / 0): 4 element ids, 4 weights\n")
        f.write("# written by make_golden.py from oracle/\n")
        for e, w in zip(cub.elem, cub.weight):
            f.write(" ".join(str(int(q)) for q in e) + " " + " ".join(f"{q:.17e}" for q in w) + "\n")
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub, REL_TOL, MAX_SWEEPS)
    write_step(os.path.join(HERE, "cube_jgs2_step.txt"),
               "JGS2 step of the 384-tet cube (Sec. 3, Sec. 5 cubature, asm correction, line search)", o)
    oj = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, REL_TOL, MAX_SWEEPS)
    write_step(os.path.join(HERE, "cube_jacobi_step.txt"),
               "uncorrected per-vertex Newton (Jacobi) step of the 384-tet cube, line search", oj)


if __name__ == "__main__":
    main()
