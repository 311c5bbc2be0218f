"""The seeded synthetic inputs follow their stated recipes (the workloads the paper's
scenes are replaced by): sizes, pinning, materials, velocities, placement and, for the
blobs, the tet-count target. The seeds are fixed, so these are exact."""
import numpy as np
import pytest

import scenes


def test_cube():
    s = scenes.cube_scene()
    assert (s.n_vertices, s.n_tets) == (125, 384)
    assert s.pinned.sum() == 25 and np.all(s.X[s.pinned.astype(bool), 2] == s.X[:, 2].max())
    assert np.allclose(s.X.max(0) - s.X.min(0), 0.1)
    assert np.all(s.youngs == 1e5) and np.all(s.poisson == 0.4) and np.all(s.density == 1000.0)
    assert np.all(s.v0 == 0.0) and s.dt == 1.0 / 120.0


def test_beam():
    s = scenes.beam_scene()
    assert (s.n_vertices, s.n_tets) == (40_000, 19 * 19 * 99 * 6)
    assert np.allclose(s.X.max(0) - s.X.min(0), [0.1, 0.02, 0.02])
    pin = s.pinned.astype(bool)
    assert pin.sum() == 400 and np.all(s.X[pin, 0] == 0.0)
    assert np.all(s.youngs == 1e7) and np.all(s.poisson == 0.45)
    assert np.all(s.v0[pin] == 0.0)
    assert abs(s.v0[~pin].std() - 0.05) < 0.001 and abs(s.v0[~pin].mean()) < 0.001


def test_ten_spheres():
    s = scenes.spheres_scene()
    assert (s.n_vertices, s.n_tets) == (634_130, 3_471_360)
    n, t = s.n_vertices // 10, s.n_tets // 10
    assert (n, t) == (63_413, 347_136)
    X = s.X.reshape(10, n, 3)
    c = X.mean(1)
    assert np.all(c >= [0.15, 0.15, 0.5]) and np.all(c <= [0.85, 0.85, 1.9])
    d = np.linalg.norm(c[:, None] - c[None], axis=2) + 10 * np.eye(10)
    assert d.min() >= 2 * 0.1 + 2 * s.dhat
    assert np.all(s.youngs[:5 * t] == 2e6) and np.all(s.youngs[5 * t:] == 1e5)
    assert s.contact == 1 and s.dhat == 1e-3 and len(s.planes) == 5
    for pl in s.planes:  # every vertex inside the box, well away from the walls
        assert (s.X @ pl[:3] - pl[3]).min() > 10 * s.dhat
    assert not s.pinned.any() and np.all(s.v0 == 0.0)


def test_blobs_hit_their_tet_targets():
    for i in range(8):
        s = scenes.blob_scene(i)
        target = scenes.blob_tet_target(i)
        assert 1e3 <= target <= 5e4
        assert abs(s.n_tets - target) <= 0.1 * target
        pin = s.pinned.astype(bool)
        assert pin.any() and np.all(np.isclose(s.X[pin, 2], s.X[:, 2].min()))
        assert 1e4 <= s.youngs[0] <= 1e7 and 0.3 <= s.poisson[0] <= 0.48


def test_contact_scenes():
    """The small contact scenes: free blocks inside the box's walls, within or just beyond
    the barrier's reach of the floor, with the stated motions."""
    d = scenes.drop_scene()
    assert len(d.X) == 64 and d.pinned.sum() == 0 and d.contact == 1
    assert d.X[:, 2].min() == pytest.approx(5e-4) and np.all(d.v0[:, 2] == -0.3)
    s = scenes.slide_scene()
    assert len(s.X) == 27 and s.X[:, 2].min() == pytest.approx(9.8e-4) and s.X[:, 2].min() < s.dhat
    assert np.all(s.v0[:, 0] == 0.5) and np.all(s.v0[:, 1] == pytest.approx(0.2))
    k = scenes.stack_scene()
    n = len(k.X) // 2
    assert len(k.X) == 54 and np.all(k.v0[:n] == 0.0) and np.all(k.v0[n:, 2] == -0.3)
    # the lower block rests 0.8 dhat above the floor, the upper one starts 0.7 mm above it
    assert k.X[:n, 2].min() == pytest.approx(0.8 * k.dhat)
    assert k.X[n:, 2].min() - k.X[:n, 2].max() == pytest.approx(0.7e-3)
    for sc in (d, s, k):
        P = sc.planes
        assert np.allclose(np.linalg.norm(P[:, :3], axis=1), 1.0)
        assert np.all(sc.X @ P[:, :3].T - P[:, 3] > 0)  # strictly inside every wall


def test_cloths():
    """Cloth grids: n x n vertices, 2 (n - 1)^2 triangles of equal area on the square, two
    adjacent corners held; the floor cloth is free and just above its wall."""
    c = scenes.cloth_scene(n=11)
    assert len(c.X) == 121 and len(c.tris) == 200
    e1 = c.X[c.tris[:, 1]] - c.X[c.tris[:, 0]]
    e2 = c.X[c.tris[:, 2]] - c.X[c.tris[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)
    assert np.allclose(area, 0.5 * 0.05 ** 2) and area.sum() == pytest.approx(0.25)
    assert list(np.nonzero(c.pinned)[0]) == [0, 110]
    f = scenes.cloth_floor_scene()
    assert f.pinned.sum() == 0 and f.X[:, 2].min() == pytest.approx(6e-4) and f.X[:, 2].min() < f.dhat
