"""Kernel timing (profile = 1) leaves the step's arithmetic alone and samples one sweep
(the last) per replayed chunk of the sweep graph: the profiled step returns the same
state, bit for bit, as the plain one, and its report counts the sampled sweeps."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [p.FP32, p.FP64])
def test_profiled_step_equals_plain_step(cuda, prec):
    import torch
    s = scenes.cube_scene()
    g = p.Mesh.from_scene(s)
    g.precompute_import(*scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=3, w_max=0.5, u_sigma=0.2))
    out = []
    for prof in (0, 1):
        x = torch.tensor(s.X, dtype=torch.float64, device=cuda)
        v = torch.tensor(s.v0, dtype=torch.float64, device=cuda)
        # rel_tol out of reach: the step runs to the cap, sweeps 0..100
        rep = g.step(x, v, p.step_opts(precision=prec, max_sweeps=100, rel_tol=1e-12, check_every=16,
                                       profile=prof))
        out.append((x.cpu().numpy(), v.cpu().numpy(), rep.sweeps, rep.launches, rep.profiled_sweeps,
                    np.array(rep.kernel_ms[:])))
    (x0, v0, k0, l0, ps0, _), (x1, v1, k1, l1, ps1, kms) = out
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    assert k0 == k1 and l0 == l1
    assert ps0 == 0
    assert k1 == 100
    assert ps1 == (k1 + 1) // 16  # replays whose last (timed) sweep ran before the stop
    names = p.jgs2.KERNEL_NAMES
    for kind in ("k_elem", "k_gather", "k_correct", "k_energy", "k_update", "setup"):
        assert kms[names.index(kind)] > 0.0, kind


def test_alu_peak_is_measured(cuda):
    """jgs2_alu_peak: FMA throughput of the CUDA cores (the ALU roofline's denominator), with
    FP32 far above FP64 on this part."""
    f32 = p.alu_peak(p.FP32)
    f64 = p.alu_peak(p.FP64)
    assert 1e3 < f32 < 2e5 and 10.0 < f64 < f32 / 4
