"""GPU test of jgs2_energy_gradient_static, the entry point for callers that cannot
allocate device memory while they run (a real-time loop that must not wait on cudaMalloc,
or a process whose device memory belongs to a pooling allocator).

It is called through the C ABI and compared with jgs2_energy_gradient, the allocating
entry point it mirrors, on two calls in a row (the calls share one static scratch array).
This file sorts last so a stop-at-first-failure run has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes

pytestmark = pytest.mark.gpu


def test_static_energy_gradient_matches_allocating_entry(cuda):
    import torch
    L = p.lib()
    L.jgs2_energy_gradient_static.argtypes = [C.c_void_p] * 7
    L.jgs2_energy_gradient_static.restype = C.c_int
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
        assert abs(E.value - E_ref) <= 1e-12 * abs(E_ref)
        gr = g_ref.cpu().numpy()
        assert np.abs(g.cpu().numpy() - gr).max() <= 1e-12 * np.abs(gr).max()


def test_static_entry_rejects_meshes_without_device_buffers(cuda):
    L = p.lib()
    L.jgs2_energy_gradient_static.argtypes = [C.c_void_p] * 7
    L.jgs2_energy_gradient_static.restype = C.c_int
    import torch
    s = scenes.cube_scene()
    mesh = p.Mesh.from_scene(s)  # no device call yet: buffers do not exist
    xt = torch.tensor(s.X, dtype=torch.float64, device=cuda)
    E = C.c_double()
    st = L.jgs2_energy_gradient_static(mesh.handle, C.c_void_p(xt.data_ptr()), C.c_void_p(xt.data_ptr()),
                                       C.c_void_p(xt.data_ptr()), C.byref(E), None, None)
    assert st == 1 and b"first" in L.jgs2_last_error()
