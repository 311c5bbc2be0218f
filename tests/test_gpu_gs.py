"""The GPU Gauss-Seidel step (jgs2_step_gs, Sec. 8.1) against the oracle's (oracle/gs.py) on
the 384-tet cube. Both sides use the same greedy colouring and the same group cubature
records, which the GPU imports. The GPU runs the colours as graph-captured passes of the
sweep kernels, each with the colour's vertex mask. They are compared after four GS sweeps
(32 colour passes): FP64 positions to 1e-9 of the step's displacement and the residual trace
to 1e-7; FP32 positions per vertex to 1e-4 of the largest vertex displacement."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, gs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("corr", [p.CORR_ASM, p.CORR_OFF])
def test_gs_step_fp64_matches_oracle(cuda, corr):
    import torch
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    col = gs.greedy_colouring(m)
    cub = gs.train_cubature_gs(m, s.dt, col) if corr == p.CORR_ASM else None
    g = p.Mesh.from_scene(s)
    if cub is not None:
        g.precompute_import(cub.elem, cub.weight, cub.ubar)
    x = torch.tensor(s.X, dtype=torch.float64, device=cuda)
    v = torch.tensor(s.v0, dtype=torch.float64, device=cuda)
    rep = g.step_gs(x, v, p.step_opts(precision=p.FP64, correction=corr, max_sweeps=4, rel_tol=1e-12,
                                      record_trace=1))
    o = gs.gs_step(m, s.X, s.v0, s.dt, s.gravity, col, cub, rel_tol=1e-12, max_sweeps=4)
    assert rep.sweeps == o.sweeps == 4 and rep.converged == 0 and not o.converged
    assert np.allclose(np.array(rep.trace[:rep.trace_len]), o.residuals, rtol=1e-7, atol=1e-12)
    d = o.x - s.X
    assert np.linalg.norm(x.cpu().numpy() - o.x) <= 1e-9 * np.linalg.norm(d)
    assert np.linalg.norm(v.cpu().numpy() - o.v) <= 1e-9 * np.linalg.norm(o.v)


@pytest.mark.parametrize("corr", [p.CORR_ASM, p.CORR_OFF])
def test_gs_step_fp32_matches_oracle(cuda, corr):
    import torch
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    col = gs.greedy_colouring(m)
    cub = gs.train_cubature_gs(m, s.dt, col) if corr == p.CORR_ASM else None
    g = p.Mesh.from_scene(s)
    if cub is not None:
        g.precompute_import(cub.elem, cub.weight, cub.ubar)
    x = torch.tensor(s.X, dtype=torch.float64, device=cuda)
    v = torch.tensor(s.v0, dtype=torch.float64, device=cuda)
    rep = g.step_gs(x, v, p.step_opts(precision=p.FP32, correction=corr, max_sweeps=4, rel_tol=1e-12))
    o = gs.gs_step(m, s.X, s.v0, s.dt, s.gravity, col, cub, rel_tol=1e-12, max_sweeps=4)
    assert rep.sweeps == o.sweeps == 4
    d = np.linalg.norm(o.x - s.X, axis=1).max()
    assert np.linalg.norm(x.cpu().numpy() - o.x, axis=1).max() <= 1e-4 * d
