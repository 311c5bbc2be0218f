"""Batched scenes (one mesh, per-scene stopping, graph-captured sweep chunks) against the
oracle run scene by scene and against single-scene GPU steps.

The batch holds three cubes of different stiffness that converge after different sweep
counts, and a beam and a blob that do not converge within the sweep cap: per-scene stopping
freezes each converged scene while the others keep sweeping.
"""
import dataclasses

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute, sweep

pytestmark = pytest.mark.gpu

CAP = 300
TOL = 1e-4


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


@pytest.fixture(scope="module")
def batch():
    cube = scenes.cube_scene()
    ss = [dataclasses.replace(cube, youngs=np.full(cube.n_tets, E)) for E in (5e4, 1e5, 2e5)]
    ss += [scenes.small_beam_scene(9, 3, 3, E=5e5, seed=3), scenes.blob_scene(7, 600, 1500)]
    ms = [fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned) for s in ss]
    cubs = [precompute.train_cubature(m, s.dt) for m, s in zip(ms, ss)]
    outs = [sweep.step(m, s.X, s.v0, s.dt, s.gravity, c, TOL, CAP) for s, m, c in zip(ss, ms, cubs)]
    return ss, ms, cubs, outs


def concat_cub(ss, cubs):
    off = np.cumsum([0] + [s.n_tets for s in ss[:-1]])
    elem = np.concatenate([np.where(c.elem >= 0, c.elem + o, -1) for c, o in zip(cubs, off)])
    return elem, np.concatenate([c.weight for c in cubs]), np.concatenate([c.ubar for c in cubs])


def test_batch_scenes_stop_independently(batch):
    ss, ms, cubs, outs = batch
    sweeps = [o.sweeps for o in outs]
    assert [o.converged for o in outs] == [True, True, True, False, False]
    assert len(set(sweeps[:3])) == 3 and sweeps[3] == sweeps[4] == CAP


@pytest.mark.parametrize("bs,persistent", [(None, 0), (64, 0), (256, 0), (None, 1), (256, 1)])
def test_batch_fp64_matches_oracle_per_scene(cuda, batch, bs, persistent):
    """Per-kernel launches (persistent 0) and the persistent cooperative launch (1): every
    scene stops at the oracle's sweep with the oracle's positions."""
    ss, ms, cubs, outs = batch
    g = p.Mesh.batch(ss)
    g.precompute_import(*concat_cub(ss, cubs))
    X = np.concatenate([s.X for s in ss])
    V0 = np.concatenate([s.v0 for s in ss])
    x, v = t(X, cuda), t(V0, cuda)
    opts = p.step_opts(precision=p.FP64, max_sweeps=CAP, rel_tol=TOL, check_every=8, persistent=persistent)
    if bs is not None:
        chosen = g.autotune(x, v, opts)
        assert chosen in (64, 128, 256)
    rep = g.step(x, v, opts)
    sw, cv, rr = g.batch_report()
    xo_all = x.cpu().numpy()
    off = 0
    for k, (s, o) in enumerate(zip(ss, outs)):
        assert cv[k] == int(o.converged), (k, cv[k], o.converged)
        assert sw[k] == o.sweeps, (k, sw[k], o.sweeps)
        xg = xo_all[off:off + s.n_vertices]
        assert np.linalg.norm(xg - o.x) <= 1e-9 * np.linalg.norm(o.x - s.X), k
        off += s.n_vertices
    assert rep.sweeps == max(sw)
    assert rep.converged == 0


def test_batch_equals_single_scene_steps(cuda, batch):
    ss, ms, cubs, outs = batch
    g = p.Mesh.batch(ss)
    g.precompute_import(*concat_cub(ss, cubs))
    X = np.concatenate([s.X for s in ss])
    V0 = np.concatenate([s.v0 for s in ss])
    xb, vb = t(X, cuda), t(V0, cuda)
    opts = p.step_opts(precision=p.FP32, max_sweeps=CAP, rel_tol=TOL)
    g.step(xb, vb, opts)
    sw, cv, _ = g.batch_report()
    off = 0
    for k, (s, c) in enumerate(zip(ss, cubs)):
        gs = p.Mesh.from_scene(s)
        gs.precompute_import(c.elem, c.weight, c.ubar)
        x, v = t(s.X, cuda), t(s.v0, cuda)
        r = gs.step(x, v, opts)
        assert r.converged == cv[k], k
        if not r.converged:
            assert r.sweeps == sw[k] == CAP
            off += s.n_vertices
            continue
        # FP32 atomics (batch) vs fixed-order block sums (single scene) change rounding, and
        # late line-search decisions with it: sweep counts agree only approximately
        assert abs(r.sweeps - sw[k]) <= max(4, r.sweeps // 4), (k, r.sweeps, sw[k])
        xs = xb.cpu().numpy()[off:off + s.n_vertices]
        assert np.linalg.norm(xs - x.cpu().numpy()) <= 1e-3 * np.linalg.norm(x.cpu().numpy() - s.X)
        off += s.n_vertices


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_fp32_matches_oracle_per_scene(cuda, batch, persistent):
    """The FP32 batch against the FP64 oracle scene by scene: every scene runs exactly 6
    sweeps (a tolerance out of reach, a cap of 6) with its own line search; per scene, the
    largest vertex error is at most 1e-4 of the largest vertex displacement."""
    ss, ms, cubs, outs = batch
    g = p.Mesh.batch(ss)
    g.precompute_import(*concat_cub(ss, cubs))
    X = np.concatenate([s.X for s in ss])
    V0 = np.concatenate([s.v0 for s in ss])
    x, v = t(X, cuda), t(V0, cuda)
    g.step(x, v, p.step_opts(precision=p.FP32, max_sweeps=6, rel_tol=1e-14, check_every=3, persistent=persistent))
    sw, _, _ = g.batch_report()
    xg_all = x.cpu().numpy()
    off = 0
    for k, (s, m, c) in enumerate(zip(ss, ms, cubs)):
        o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, c, 1e-14, 6)
        assert sw[k] == o.sweeps == 6
        xg = xg_all[off:off + s.n_vertices]
        err = np.linalg.norm(xg - o.x, axis=1).max() / np.linalg.norm(o.x - s.X, axis=1).max()
        assert err <= 1e-4, (k, err)
        off += s.n_vertices


def test_persistent_barrier_wait_runs_out(cuda, batch):
    """A bounded device wait that runs out: the test hook makes the persistent launch's first
    grid barrier wait for one block more than the grid has, with a short wait limit set from
    the host. Every block gives up after its polls, the step returns JGS2_ETIMEOUT with the
    state not written, and the next step on the same mesh runs normally."""
    ss, ms, cubs, outs = batch
    g = p.Mesh.batch(ss)
    g.precompute_import(*concat_cub(ss, cubs))
    X = np.concatenate([s.X for s in ss])
    V0 = np.concatenate([s.v0 for s in ss])
    x, v = t(X, cuda), t(V0, cuda)
    hook = p.step_opts(precision=p.FP32, max_sweeps=CAP, rel_tol=TOL, persistent=1, wait_polls=2000,
                       test_unreachable_barrier=1)
    with pytest.raises(p.JGS2Error) as ei:
        g.step(x, v, hook)
    assert ei.value.status == 8
    assert np.array_equal(x.cpu().numpy(), X) and np.array_equal(v.cpu().numpy(), V0)
    rep = g.step(x, v, p.step_opts(precision=p.FP32, max_sweeps=CAP, rel_tol=TOL, persistent=1))
    assert rep.sweeps > 0 and np.isfinite(x.cpu().numpy()).all()
