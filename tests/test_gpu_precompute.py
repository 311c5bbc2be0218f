"""The precompute with its multi-RHS solves on the GPU (jgs2_precompute_opts.gpu = 1: FP32
supernodal substitutions refined in FP64 against H_bar) against the host's FP64
substitutions (gpu = 0), which tests/test_precompute_parity.py pins to the oracle (Secs. 5-6).

The refined solves reach a relative residual of 1e-14, so the training poses and the rows
of H_bar^{-1} agree with the host's to about kappa(H_bar) 1e-14: on the cube and the beam
the greedy sets (Eq. cubature_weight) are identical, and weights, U_bar rows (Eq. u) and fit
residuals agree to 1e-7 relative (1e-6 on the free sphere, whose mass-only lowest modes
make H_bar the worst conditioned). The sphere is large enough that the top separator's
panels have more than 256 rows below them, so the split forward updates and the backward
partial sums run."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes

pytestmark = pytest.mark.gpu


def both(s, **kw):
    out = []
    for gpu in (0, 1):
        g = p.Mesh.from_scene(s)
        g.precompute(gpu=gpu, **kw)
        out.append(g.precompute_export())
        g.close()
    return out


def check(host, dev, free, rtol):
    (e0, w0, u0, r0), (e1, w1, u1, r1) = host, dev
    assert np.array_equal(e0, e1)
    assert np.max(np.abs(w1 - w0)) <= rtol * max(np.max(np.abs(w0)), 1e-300)
    assert np.max(np.abs(u1 - u0)) <= rtol * np.max(np.abs(u0))
    assert np.allclose(r1[free], r0[free], rtol=rtol, atol=1e-12)


def test_gpu_precompute_cube(cuda):
    s = scenes.cube_scene()
    check(*both(s, n_cub=4), ~s.pinned.astype(bool), 1e-9)


def test_gpu_precompute_stiff_beam(cuda):
    s = scenes.small_beam_scene(nvx=21, nvy=6, nvz=6, E=1e7)
    check(*both(s, n_cub=4), ~s.pinned.astype(bool), 1e-7)


def test_gpu_precompute_free_sphere(cuda):
    # free-floating (no pins): H_bar's smallest eigenvalues are the mass term's alone. The
    # rest positions are jittered by a seeded 5 % of a cell, which breaks the voxel sphere's
    # symmetry: a symmetric body has eigenvalues of multiplicity 2-3 whose eigenvectors are
    # any basis of their eigenspace, so rounding would pick the training poses.
    X, tets = scenes.voxel_sphere(0.1, 24)
    X = X + np.random.default_rng(7).uniform(-1.0, 1.0, X.shape) * 0.05 * (0.2 / 24)
    T = len(tets)
    s = scenes.Scene("sphere24", X, tets.astype(np.int32), np.full(T, 2e6), np.full(T, 0.4),
                     np.full(T, 1000.0), np.zeros(len(X), np.uint8), np.zeros_like(X))
    check(*both(s, n_cub=4), np.ones(len(X), bool), 1e-6)
