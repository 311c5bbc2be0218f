"""The library's host precompute (jgs2_precompute: FP64 C++ on the host, no GPU needed)
against the oracle's (Secs. 5-6). The U_bar rows it exports equal the oracle's Eq. u rows
at the same elements' corners. The greedy NNLS sets (Eq. cubature_weight) with their
weights and fit residuals equal the oracle's wherever both saw the same training poses.
On the cube that is every vertex. Elsewhere, eigenvectors of repeated eigenvalues can be
any basis of their eigenspace, so a few vertices may legitimately pick other elements.
Weights and residuals agree to 1e-6: the library's training poses come from block inverse
iteration, stopped at a relative eigen-residual of 1e-8, and the oracle's from a dense
eigensolver."""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute


def lib_precompute(s):
    g = p.Mesh.from_scene(s)
    g.precompute(n_cub=4)
    out = g.precompute_export()
    g.close()
    return out


def test_cube_precompute_matches_oracle():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    cub = precompute.train_cubature(m, s.dt)
    e, w, u, r = lib_precompute(s)
    free = ~s.pinned.astype(bool)
    assert np.array_equal(e, cub.elem)
    assert np.allclose(w, cub.weight, rtol=1e-6, atol=1e-9)
    assert np.max(np.abs(u - cub.ubar)) <= 1e-12 * np.max(np.abs(cub.ubar))
    assert np.allclose(r[free], cub.residual[free], rtol=1e-6, atol=1e-9)


def test_beam_precompute_ubar_rows_and_sets():
    s = scenes.small_beam_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    Hbar = precompute.rest_hessian(m, s.dt)
    Ub, _ = precompute.ubar_all(m, Hbar)
    cub = precompute.train_cubature(m, s.dt, Hbar=Hbar)
    e, w, u, r = lib_precompute(s)
    free = np.nonzero(~s.pinned.astype(bool))[0]
    scale = np.max(np.abs(Ub))
    # every exported U_bar block is the oracle's Eq. u row of that corner (zero if pinned)
    n_checked = 0
    for i in free:
        di = m.dof_of[i]
        for k in range(e.shape[1]):
            if e[i, k] < 0:
                continue
            for c, a in enumerate(s.tets[e[i, k]]):
                da = m.dof_of[a]
                ref = np.zeros((3, 3)) if da < 0 else Ub[di][3 * da:3 * da + 3]
                assert np.max(np.abs(u[i, k, c] - ref)) <= 1e-12 * scale
                n_checked += 1
    assert n_checked > 3 * len(free)
    same = np.all(e[free] == cub.elem[free], axis=1)
    assert same.mean() >= 0.95
    rows = free[same]
    assert np.allclose(w[rows], cub.weight[rows], rtol=1e-6, atol=1e-9)
    assert np.allclose(r[rows], cub.residual[rows], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("name", ["cube", "beam"])
def test_gs_group_precompute_matches_oracle(name):
    """jgs2_precompute with gs = 1 (Sec. 8.1 groups) against oracle/gs.py: every exported
    U_bar block is the oracle's group U_bar row (zero inside the group), and the greedy
    sets, weights and residuals agree wherever both picked the same elements."""
    from oracle import gs
    s = scenes.cube_scene() if name == "cube" else scenes.small_beam_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    col = gs.greedy_colouring(m)
    Hbar = precompute.rest_hessian(m, s.dt)
    Ub = gs.ubar_groups(m, Hbar, col)
    cub = gs.train_cubature_gs(m, s.dt, col, Hbar=Hbar)
    g = p.Mesh.from_scene(s)
    g.precompute(n_cub=4, gs=1)
    e, w, u, r = g.precompute_export()
    g.close()
    free = np.nonzero(~s.pinned.astype(bool))[0]
    scale = np.max(np.abs(Ub))
    for i in free:
        di = m.dof_of[i]
        for k in range(e.shape[1]):
            if e[i, k] < 0:
                continue
            for c, a in enumerate(s.tets[e[i, k]]):
                da = m.dof_of[a]
                ref = np.zeros((3, 3)) if da < 0 else Ub[di][3 * da:3 * da + 3]
                assert np.max(np.abs(u[i, k, c] - ref)) <= 1e-12 * scale
    same = np.all(e[free] == cub.elem[free], axis=1)
    assert same.mean() >= 0.95
    rows = free[same]
    assert np.allclose(w[rows], cub.weight[rows], rtol=1e-5, atol=1e-8)
    assert np.allclose(r[rows], cub.residual[rows], rtol=1e-5, atol=1e-8)


def test_precompute_gpu_option_range():
    # validated before any work: 0 (host solves) or 1 (GPU solves)
    g = p.Mesh.from_scene(scenes.cube_scene())
    with pytest.raises(p.JGS2Error):
        g.precompute(gpu=2)
    g.close()


def test_batch_precompute_matches_each_scene_alone():
    """A mesh of several scenes precomputes each body on its own: the bodies of a batch run
    side by side (one thread each) and must give the cubature each scene gets alone: the
    same element sets, and weights, U_bar rows and residuals equal to rounding (a scene of
    one body runs it on all threads, which splits its pool solves into column chunks)."""
    idx = [24, 35, 18, 8]  # four small seeded blobs (1-2k tets)
    ss = [scenes.blob_scene(i) for i in idx]
    g = p.Mesh.batch(ss)
    g.precompute(n_cub=4)
    e, w, u, r = g.precompute_export()
    # several small bodies take the host path side by side even when GPU solves are asked
    # for (so this runs without a device too), with the same results
    g.precompute(n_cub=4, gpu=1)
    for a, b in zip((e, w, u, r), g.precompute_export()):
        assert np.array_equal(a, b, equal_nan=a.dtype.kind == "f")
    g.close()
    v0 = t0 = 0  # the batch numbers vertices and tets scene after scene
    for s in ss:
        es, ws, us, rs = lib_precompute(s)
        nv = len(s.X)
        free = ~s.pinned.astype(bool)
        eb = e[v0:v0 + nv][free]
        assert np.array_equal(np.where(eb >= 0, eb - t0, -1), es[free])
        assert np.allclose(w[v0:v0 + nv][free], ws[free], rtol=1e-9, atol=1e-12 * np.abs(ws).max())
        assert np.max(np.abs(u[v0:v0 + nv][free] - us[free])) <= 1e-9 * np.abs(us).max()
        assert np.allclose(r[v0:v0 + nv][free], rs[free], rtol=1e-7, atol=1e-12)
        v0 += nv
        t0 += len(s.tets)


def test_precompute_does_not_depend_on_the_thread_count():
    """The host precompute's tree passes run level by level in parallel; a supernode's
    arithmetic does not depend on the schedule, so one thread and several give the same
    cubature sets, and values equal to rounding (the pool solves split their columns into
    one chunk per thread)."""
    s = scenes.small_beam_scene(nvx=21, nvy=6, nvz=6, E=1e7)  # 756 vertices, a deeper tree
    outs = []
    for nt in (1, 4):
        g = p.Mesh.from_scene(s)
        g.precompute(n_cub=4, n_threads=nt)
        outs.append(g.precompute_export())
        g.close()
    (e1, w1, u1, r1), (e4, w4, u4, r4) = outs
    free = ~s.pinned.astype(bool)
    assert np.array_equal(e1, e4)
    assert np.allclose(w1[free], w4[free], rtol=1e-9, atol=1e-12 * np.abs(w1).max())
    assert np.max(np.abs(u1 - u4)) <= 1e-10 * np.abs(u1).max()
    assert np.allclose(r1[free], r4[free], rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("name", ["cube", "beam"])
def test_cubature_import_export_round_trip(name):
    """jgs2_precompute_import takes records in the caller's vertex and tet order and stores
    them in the library's (Morton-ordered vertices, sorted tets); the export maps them back.
    The round trip is exact for free vertices; pinned vertices export empty slots."""
    s = scenes.cube_scene() if name == "cube" else scenes.small_beam_scene(nvx=21, nvy=6, nvz=6, E=1e7)
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    cub = precompute.train_cubature(m, s.dt)
    g = p.Mesh.from_scene(s)
    g.precompute_import(cub.elem, cub.weight, cub.ubar)
    e, w, u, _ = g.precompute_export()
    g.close()
    free = ~s.pinned.astype(bool)
    assert np.array_equal(e[free], cub.elem[free])
    assert np.array_equal(w[free], cub.weight[free])
    assert np.array_equal(u[free], cub.ubar[free])
    assert np.all(e[~free] == -1) and np.all(w[~free] == 0.0)
