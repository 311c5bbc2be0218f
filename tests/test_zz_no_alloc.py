"""Tests of jgs2_energy_gradient_static, the entry point for callers that cannot allocate
device memory while they run (a real-time loop that must not wait on cudaMalloc, or a
process whose device memory belongs to a pooling allocator).

The GPU tests call it through the C ABI and compare it with jgs2_energy_gradient, the
allocating entry point it mirrors, on two calls in a row (the calls share one static
scratch array). Its input checks (contact meshes, meshes beyond the scratch size) run
before any device work, so they are tested on the host. This file sorts last so a
stop-at-first-failure run has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes

STATIC_PARTIALS_MAX = 65536   # JGS2_STATIC_PARTIALS_MAX in include/jgs2.h


def _static_fn():
    L = p.lib()
    L.jgs2_energy_gradient_static.argtypes = [C.c_void_p] * 7
    L.jgs2_energy_gradient_static.restype = C.c_int
    return L


def _call_with_dummy_pointers(L, mesh):
    """Calls the entry point with non-null stand-ins for the device arrays: valid for the
    input checks that reject the call before any device work."""
    buf = (C.c_double * 3)()
    E = C.c_double()
    ptr = C.cast(buf, C.c_void_p)
    return L.jgs2_energy_gradient_static(mesh.handle, ptr, ptr, ptr, C.byref(E), None, None)


@pytest.mark.gpu
def test_static_energy_gradient_matches_allocating_entry(cuda):
    import torch
    L = _static_fn()
    s = scenes.beam_scene(21, 6, 6, 0.1, 0.025, 1e6, 0.45, 0.05, seed=3)
    mesh = p.Mesh.from_scene(s)
    dev = cuda
    xt = torch.tensor(s.X, dtype=torch.float64, device=dev)
    vt = torch.tensor(s.v0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    states = [scenes.perturbed_state(s.X, s.pinned, 2e-4, seed=k) for k in (7, 8)]
    # the allocating entry point creates the mesh's device buffers and gives the reference
    ref = []
    for xs in states:
        x = torch.tensor(xs, dtype=torch.float64, device=dev)
        ref.append(mesh.energy_gradient(xt, vt, x))
    for (E_ref, g_ref), xs in zip(ref, states):
        x = torch.tensor(xs, dtype=torch.float64, device=dev)
        g = torch.full_like(x, float("nan"))
        E = C.c_double(float("nan"))
        st = L.jgs2_energy_gradient_static(mesh.handle, C.c_void_p(xt.data_ptr()), C.c_void_p(vt.data_ptr()),
                                           C.c_void_p(x.data_ptr()), C.byref(E), C.c_void_p(g.data_ptr()),
                                           C.c_void_p(stream))
        assert st == 0, L.jgs2_last_error().decode()
        # E: the same partials summed in another fixed order; g: the same kernel
        assert abs(E.value - E_ref) <= 1e-12 * abs(E_ref)
        gr = g_ref.cpu().numpy()
        assert np.array_equal(g.cpu().numpy(), gr)


@pytest.mark.gpu
def test_static_entry_rejects_meshes_without_device_buffers(cuda):
    L = _static_fn()
    import torch
    s = scenes.cube_scene()
    mesh = p.Mesh.from_scene(s)  # no device call yet: buffers do not exist
    xt = torch.tensor(s.X, dtype=torch.float64, device=cuda)
    E = C.c_double()
    st = L.jgs2_energy_gradient_static(mesh.handle, C.c_void_p(xt.data_ptr()), C.c_void_p(xt.data_ptr()),
                                       C.c_void_p(xt.data_ptr()), C.byref(E), None, None)
    assert st == 1 and b"first" in L.jgs2_last_error()


def test_static_entry_rejects_contact_meshes():
    """The barrier needs the candidate list only the allocating entry point builds: a
    contact mesh is refused before any device work."""
    L = _static_fn()
    mesh = p.Mesh.from_scene(scenes.drop_scene())
    assert _call_with_dummy_pointers(L, mesh) == 1
    assert b"contact" in L.jgs2_last_error()


def test_static_entry_rejects_meshes_beyond_the_scratch_size():
    """(n_tets + free vertices) / 128 block partials must fit the static array; a
    100x100x125-vertex grid (7,291,944 tets, 1,250,000 free vertices) needs 66,729."""
    X, tets = scenes.kuhn_grid(100, 100, 125, (0.1, 0.1, 0.125))
    T = len(tets)
    nblocks = -(-T // 128) + -(-len(X) // 128)
    assert nblocks > STATIC_PARTIALS_MAX
    s = scenes.Scene("grid", X, tets, np.full(T, 1e5), np.full(T, 0.4), np.full(T, 1000.0),
                     np.zeros(len(X), np.uint8), np.zeros_like(X))
    L = _static_fn()
    mesh = p.Mesh.from_scene(s)
    assert _call_with_dummy_pointers(L, mesh) == 1
    assert b"too large" in L.jgs2_last_error()
    mesh.close()
