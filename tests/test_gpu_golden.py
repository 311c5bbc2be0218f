"""The CUDA step (FP64, through the C ABI) against the stored oracle values of
tests/golden/: the 384-tet cube's implicit-Euler step (Sec. 3) by JGS2 sweeps with the
oracle's cubature (Sec. 5) and by uncorrected Jacobi sweeps. Same tolerances as the live
parity tests: residual trace 1e-7 relative, positions 1e-9 of the step's displacement."""
import importlib.util
import os

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
golden = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(golden)


@pytest.mark.parametrize("name,corr", [("cube_jgs2_step.txt", p.CORR_ASM), ("cube_jacobi_step.txt", p.CORR_OFF)])
def test_fp64_step_matches_golden(cuda, name, corr):
    import torch
    s = scenes.cube_scene()
    sweeps, conv, res, xg = golden.load_step(os.path.join(HERE, name))
    g = p.Mesh.from_scene(s)
    if corr != p.CORR_OFF:
        m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
        cub = precompute.train_cubature(m, s.dt)
        elem, _ = golden.load_cubature(os.path.join(HERE, "cube_cubature.txt"))
        assert np.array_equal(cub.elem, elem)  # the records the fixture was made with
        g.precompute_import(cub.elem, cub.weight, cub.ubar)
    x = torch.tensor(s.X, dtype=torch.float64, device=cuda)
    v = torch.tensor(s.v0, dtype=torch.float64, device=cuda)
    rep = g.step(x, v, p.step_opts(precision=p.FP64, correction=corr, rel_tol=golden.REL_TOL,
                                   max_sweeps=golden.MAX_SWEEPS, record_trace=1))
    assert rep.sweeps == sweeps and bool(rep.converged) == conv
    assert np.allclose(np.array(rep.trace[:rep.trace_len]), res, rtol=1e-7, atol=1e-12)
    assert np.linalg.norm(x.cpu().numpy() - xg) <= 1e-9 * np.linalg.norm(xg - s.X)
