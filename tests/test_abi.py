"""The C ABI library loads, exports every symbol include/jgs2.h declares, and rejects bad
mesh descriptions before touching a GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from paper_2506_06494_b300 import jgs2 as J

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "jgs2.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(jgs2_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_2506_06494_b300 import build
    build.build()
    return p.lib()


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert "jgs2_step" in syms and "jgs2_mesh_create" in syms
    for s in syms:
        assert hasattr(L, s), s


def test_default_options(L):
    o = p.step_opts()
    assert o.max_sweeps == 500 and o.rel_tol == 1e-4 and o.precision == p.FP32
    assert o.correction == p.CORR_ASM and o.line_search == 1
    q = p.precompute_opts()
    assert q.n_cub == 4 and q.n_train == 20 and q.n_cand == 32 and q.nnls_tol == 0.01 and q.gs == 0


def _desc(X, T, E, nu, rho, pin=None, dt=1 / 120):
    d = J.MeshDesc()
    d.n_vertices = len(X)
    d.n_tets = len(T)
    d.rest_pos = X.ctypes.data_as(C.POINTER(C.c_double))
    d.tets = T.ctypes.data_as(C.POINTER(C.c_int32))
    d.youngs = E.ctypes.data_as(C.POINTER(C.c_double))
    d.poisson = nu.ctypes.data_as(C.POINTER(C.c_double))
    d.density = rho.ctypes.data_as(C.POINTER(C.c_double))
    d.pinned = C.POINTER(C.c_uint8)() if pin is None else pin.ctypes.data_as(C.POINTER(C.c_uint8))
    d.dt = dt
    return d


@pytest.mark.parametrize("case", ["inverted", "index", "material", "dt", "empty", "isolated", "friction_neg",
                                  "friction_no_contact", "friction_eps"])
def test_mesh_create_rejects_bad_input(L, case):
    s = scenes.cube_scene()
    X = s.X.copy()
    T = s.tets.astype(np.int32).copy()
    E, nu, rho = s.youngs.copy(), s.poisson.copy(), s.density.copy()
    dt = 1 / 120
    if case == "inverted":
        T[5, [1, 2]] = T[5, [2, 1]]
    elif case == "index":
        T[7, 3] = len(X)
    elif case == "material":
        nu[3] = 0.5
    elif case == "dt":
        dt = 0.0
    elif case == "isolated":  # a free vertex in no tet: no mass, singular 3x3 system
        X = np.vstack([X, [[1.0, 1.0, 1.0]]])
    d = _desc(X, T, E, nu, rho, None, dt)
    if case == "empty":
        d.n_tets = 0
    elif case == "friction_neg":
        d.friction_mu = -0.1
    elif case == "friction_no_contact":  # friction needs the walls' normal forces
        d.friction_mu, d.friction_eps_v = 0.5, 1e-3
    elif case == "friction_eps":
        d.contact, d.dhat, d.kappa = 1, 1e-3, 1e5
        d.friction_mu, d.friction_eps_v = 0.5, 0.0
    h = C.c_void_p()
    st = L.jgs2_mesh_create(C.byref(d), C.byref(h))
    assert st == 1  # JGS2_EINVAL, raised before any device allocation
    assert not h.value
    assert len(L.jgs2_last_error()) > 0


def test_pinned_vertex_outside_every_tet_is_accepted(L):
    """A pinned vertex that no tet references carries no DOF: the mesh is valid (creation
    is host-only, so this runs without a GPU)."""
    s = scenes.cube_scene()
    X = np.vstack([s.X, [[1.0, 1.0, 1.0]]])
    T = s.tets.astype(np.int32).copy()
    pin = np.zeros(len(X), np.uint8)
    pin[-1] = 1
    E, nu, rho = s.youngs.copy(), s.poisson.copy(), s.density.copy()
    d = _desc(X, T, E, nu, rho, pin)
    h = C.c_void_p()
    assert L.jgs2_mesh_create(C.byref(d), C.byref(h)) == 0
    L.jgs2_mesh_destroy(h)


def test_contact_form_is_validated(L):
    """contact = 1 (IPC barrier) and 2 (penalty) are accepted; any other value is refused
    before any device work."""
    s = scenes.drop_scene()
    X, T = np.ascontiguousarray(s.X), s.tets.astype(np.int32)   # kept alive for the call
    E, nu, rho = s.youngs.copy(), s.poisson.copy(), s.density.copy()
    planes = np.ascontiguousarray(s.planes, dtype=np.float64)
    for form, want in ((1, 0), (2, 0), (3, 1), (-1, 1)):
        d = _desc(X, T, E, nu, rho, None)
        d.contact = form
        d.n_planes = len(planes)
        d.planes = planes.ctypes.data_as(C.POINTER(C.c_double))
        d.dhat = s.dhat
        d.kappa = s.kappa
        h = C.c_void_p()
        assert L.jgs2_mesh_create(C.byref(d), C.byref(h)) == want, form
        if want == 0:
            L.jgs2_mesh_destroy(h)


def test_wall_planes_are_validated(L):
    """Wall normals must be unit vectors and offsets finite (the barrier's distance n.x - c
    assumes both)."""
    s = scenes.drop_scene()
    X, T = np.ascontiguousarray(s.X), s.tets.astype(np.int32)
    E, nu, rho = s.youngs.copy(), s.poisson.copy(), s.density.copy()
    for bad in ("scaled", "nan_offset", "zero"):
        planes = np.ascontiguousarray(s.planes, dtype=np.float64).copy()
        if bad == "scaled":
            planes[1, :3] *= 1.5
        elif bad == "nan_offset":
            planes[2, 3] = np.inf
        else:
            planes[0, :3] = 0.0
        d = _desc(X, T, E, nu, rho, None)
        d.contact = 1
        d.n_planes = len(planes)
        d.planes = planes.ctypes.data_as(C.POINTER(C.c_double))
        d.dhat = s.dhat
        d.kappa = s.kappa
        h = C.c_void_p()
        assert L.jgs2_mesh_create(C.byref(d), C.byref(h)) == 1, bad


def test_null_arguments(L):
    h = C.c_void_p()
    assert L.jgs2_mesh_create(None, C.byref(h)) == 1
    assert L.jgs2_step(None, None, None, None, None, None) == 1
    assert L.jgs2_precompute_import(None, None) == 1


def test_batch_create_validates_scenes(L):
    """jgs2_mesh_create_batch (host-only, no GPU): scenes must share dt and gravity, and a
    batch carries no contact."""
    a, b = scenes.cube_scene(), scenes.cube_scene()
    m = p.Mesh.batch([a, b])  # valid: two scenes
    assert m.n_scenes == 2 and m.V == 2 * a.n_vertices
    m.close()
    b.dt = a.dt / 2
    with pytest.raises(p.JGS2Error):
        p.Mesh.batch([a, b])
    b = scenes.cube_scene()
    b.gravity = (0.0, 0.0, -1.0)
    with pytest.raises(p.JGS2Error):
        p.Mesh.batch([a, b])
    keep = []
    descs = (J.MeshDesc * 2)()
    for k, s in enumerate([a, scenes.cube_scene()]):
        descs[k] = J._desc(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned, s.gravity, s.dt,
                           None, 1e-3, 1e4, 1 if k == 1 else 0, keep)
    h = C.c_void_p()
    assert L.jgs2_mesh_create_batch(descs, 2, C.byref(h)) == 1  # JGS2_EINVAL
    assert not h.value


@pytest.mark.parametrize("bad", [np.nan, 0.0, -1e5, np.inf])
def test_poisoned_youngs_modulus_is_rejected(L, bad):
    """jgs2_mesh_set_youngs validates every modulus before it changes anything (host-only
    before the mesh reaches a device)."""
    s = scenes.cube_scene()
    g = p.Mesh.from_scene(s)
    E = np.full(s.n_tets, 1e5)
    E[17] = bad
    with pytest.raises(p.JGS2Error) as err:
        g.set_youngs(E)
    assert err.value.status == 1
    g.set_youngs(np.full(s.n_tets, 2e5))  # a valid set is accepted
    g.close()


def test_gs_step_rejects_contact_and_batches(L):
    """jgs2_step_gs takes single scenes without contact; the check comes before any device
    work, so dummy host pointers never reach a kernel."""
    dummy = np.zeros(3)
    ptr = dummy.ctypes.data_as(C.c_void_p)
    opts = p.step_opts(correction=p.CORR_OFF)
    drop = p.Mesh.from_scene(scenes.drop_scene())
    assert L.jgs2_step_gs(drop.handle, ptr, ptr, C.byref(opts), None, None) == 1  # JGS2_EINVAL
    drop.close()
    batch = p.Mesh.batch([scenes.cube_scene(), scenes.cube_scene()])
    assert L.jgs2_step_gs(batch.handle, ptr, ptr, C.byref(opts), None, None) == 1
    batch.close()


@pytest.mark.parametrize("case", ["index", "degenerate", "material", "dt", "isolated"])
def test_cloth_create_rejects_bad_input(case):
    s = scenes.cloth_scene(n=4)
    X, T = s.X.copy(), s.tris.copy()
    kw = dict(youngs=s.youngs, poisson=s.poisson, thickness=s.thickness, density=s.density, bend=s.bend, dt=s.dt)
    if case == "index":
        T[3, 1] = len(X)
    elif case == "degenerate":
        T[2, 2] = T[2, 1]
    elif case == "material":
        kw["poisson"] = 0.5
    elif case == "dt":
        kw["dt"] = 0.0
    elif case == "isolated":
        X = np.vstack([X, [[2.0, 2.0, 0.0]]])
    with pytest.raises(J.JGS2Error):
        J.Cloth(X, T, kw["youngs"], kw["poisson"], kw["thickness"], kw["density"], kw["bend"], None,
                dt=kw["dt"])


@pytest.mark.parametrize("case", ["normal", "offset", "behind", "on"])
def test_cloth_walls_are_validated(case):
    s = scenes.cloth_floor_scene(n=4)
    X, planes = s.X.copy(), s.planes.copy()
    want = 1  # JGS2_EINVAL
    if case == "normal":
        planes[0, :3] *= 2.0
    elif case == "offset":
        planes[0, 3] = np.nan
    elif case == "behind":
        X[5, 2] = -1e-4
        want = 9  # JGS2_EINTERSECT: a free rest vertex behind the floor
    elif case == "on":
        X[5, 2] = 0.0
        want = 9
    with pytest.raises(J.JGS2Error) as e:
        J.Cloth(X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, s.pinned, dt=s.dt,
                planes=planes, dhat=s.dhat, kappa=s.kappa)
    assert e.value.status == want
    # a pinned vertex may sit anywhere
    if case in ("behind", "on"):
        pin = s.pinned.copy()
        pin[5] = 1
        c = J.Cloth(X, s.tris, s.youngs, s.poisson, s.thickness, s.density, s.bend, pin, dt=s.dt,
                    planes=planes, dhat=s.dhat, kappa=s.kappa)
        c.close()


def test_cloth_hinges_are_the_interior_edges():
    # an n x n grid cut into 2 triangles per cell has 2 n (n - 1) + (n - 1)^2 edges, 4 (n - 1)
    # of them on the boundary
    for n in (3, 8):
        s = scenes.cloth_scene(n=n)
        c = J.Cloth.from_scene(s)
        assert c.n_hinges == 2 * n * (n - 1) + (n - 1) ** 2 - 4 * (n - 1)
        c.close()

