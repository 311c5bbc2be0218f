"""GPU parity: the CUDA sweep (through the C ABI) against the FP64 oracle.

Tolerances, per vertex: max_i |x_gpu,i - x_orc,i| / max_i |x_orc,i - x_start,i| (the largest
vertex error over the largest vertex displacement of the sweeps compared) is at most 1e-9 for
the FP64 path and 1e-4 for the FP32 path. Identical precompute data goes to both sides: the
GPU gets the oracle's cubature records (or a seeded synthetic record set) through
jgs2_precompute_import.
"""
import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, local, precompute, sweep

pytestmark = pytest.mark.gpu

TOL = {p.FP64: 1e-9, p.FP32: 1e-4}
GRAD = {p.CORR_ASM: "asm", p.CORR_ELEM: "elem"}


@pytest.fixture(scope="module")
def cube():
    s = scenes.cube_scene()
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    cub = precompute.train_cubature(m, s.dt)
    return s, m, cub


@pytest.fixture(scope="module")
def beam():
    # 21x6x6 vertices: 720 free vertices = 5 full 128-vertex blocks and a ragged tail
    s = scenes.beam_scene(21, 6, 6, 0.1, 0.025, 1e6, 0.45, 0.05, seed=1)
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=2, w_max=0.5, u_sigma=0.2)
    cub = precompute.Cubature(elem, w, u, np.zeros(len(s.X)))
    return s, m, cub


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def gpu_mesh(s, cub=None):
    g = p.Mesh.from_scene(s)
    if cub is not None:
        g.precompute_import(cub.elem, cub.weight, cub.ubar)
    return g


def rel(a, b, ref):
    """Largest per-vertex error of a against b over the largest per-vertex norm of ref."""
    a, b, ref = (np.asarray(q).reshape(-1, 3) for q in (a, b, ref))
    return np.linalg.norm(a - b, axis=1).max() / max(np.linalg.norm(ref, axis=1).max(), 1e-300)


def test_energy_gradient_fp64(cuda, cube):
    s, m, _ = cube
    x = scenes.perturbed_state(s.X, s.pinned, 2e-3, seed=1)
    v = 0.1 * np.ones_like(s.X)
    g_mesh = gpu_mesh(s)
    E, g = g_mesh.energy_gradient(t(s.X, cuda), t(v, cuda), t(x, cuda))
    z = fem.inertia_target(s.X, v, s.dt, s.gravity)
    g_o = fem.vertex_gradient(m, x, z, s.dt)
    assert np.abs(g.cpu().numpy() - g_o).max() <= 1e-11 * np.abs(g_o).max()
    # energy is offset-free only up to the constant inertia of pinned vertices (none moved)
    assert abs(E - fem.energy(m, x, z, s.dt)) <= 1e-11 * abs(E)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
@pytest.mark.parametrize("corr", [p.CORR_ASM, p.CORR_ELEM, p.CORR_OFF])
@pytest.mark.parametrize("ls", [0, 1])
def test_one_sweep_cube(cuda, cube, prec, corr, ls):
    s, m, cub = cube
    xk = scenes.perturbed_state(s.X, s.pinned, 1e-3, seed=4)
    v = scenes.perturbed_state(np.zeros_like(s.X), s.pinned, 0.05, seed=5)
    gm = gpu_mesh(s, cub)
    xg = t(xk, cuda)
    gm.sweeps(t(s.X, cuda), t(v, cuda), xg, 1, p.step_opts(precision=prec, correction=corr, line_search=ls))
    z = fem.inertia_target(s.X, v, s.dt, s.gravity)
    c = None if corr == p.CORR_OFF else cub
    xo = sweep.run_sweeps(m, xk, z, s.dt, c, 1, grad=GRAD.get(corr, "asm"), line_search_on=bool(ls))
    assert rel(xg.cpu().numpy(), xo, xo - xk) <= TOL[prec]


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_three_sweeps_multiblock_beam(cuda, beam, prec):
    s, m, cub = beam
    xk = scenes.perturbed_state(s.X, s.pinned, 2e-4, seed=6)
    gm = gpu_mesh(s, cub)
    xg = t(xk, cuda)
    gm.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 3, p.step_opts(precision=prec))
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    xo = sweep.run_sweeps(m, xk, z, s.dt, cub, 3)
    assert rel(xg.cpu().numpy(), xo, xo - xk) <= TOL[prec]


def test_step_fp64_matches_oracle(cuda, cube):
    s, m, cub = cube
    gm = gpu_mesh(s, cub)
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    rep = gm.step(x, v, p.step_opts(precision=p.FP64, max_sweeps=400, record_trace=1))
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub, 1e-4, 400)
    assert rep.converged == 1 and o.converged
    assert rep.sweeps == o.sweeps
    tr = np.array(rep.trace[:rep.trace_len])
    assert np.allclose(tr, o.residuals, rtol=1e-7, atol=1e-12)
    assert rel(x.cpu().numpy(), o.x, o.x - s.X) <= 1e-9
    assert rel(v.cpu().numpy(), o.v, o.v) <= 1e-9


def test_step_position_change_stop_matches_oracle(cuda, cube):
    """Sec. 8's stopping test (|x^k - x^{k-1}| <= dx_tol L): the FP64 step stops at the
    oracle's sweep, with its positions."""
    s, m, cub = cube
    gm = gpu_mesh(s, cub)
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    rep = gm.step(x, v, p.step_opts(precision=p.FP64, max_sweeps=400, dx_tol=1e-4, length_scale=0.1))
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub, 1e-4, 400, dx_tol=1e-4, length_scale=0.1,
                   record_x=True)
    assert o.stopped_dx and not o.converged
    assert rep.stopped_dx == 1 and rep.converged == 0 and rep.sweeps == o.sweeps
    assert rel(x.cpu().numpy(), o.x, o.x - s.X) <= 1e-9
    last = np.linalg.norm((o.xs[-1] - o.xs[-2])[m.free]) / 0.1
    assert last <= 1e-4 and abs(rep.last_dx - last) <= 1e-6 * last


def test_step_fp32_converges_to_oracle_solution(cuda, cube):
    """FP32 sweeps take their own line-search path, so the step is checked by what must hold
    for any valid result: the FP64 oracle's relative residual at the GPU's x_{t+1} meets the
    1e-4 target (2x slack for FP32 rounding of the stopping test), and x_{t+1} is within the
    Newton-predicted distance H^{-1} g of the oracle's tightly converged x*."""
    s, m, cub = cube
    gm = gpu_mesh(s, cub)
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    rep = gm.step(x, v, p.step_opts(precision=p.FP32, max_sweeps=3000, rel_tol=1e-4))
    assert rep.converged == 1
    xg = x.cpu().numpy()
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    g0 = np.linalg.norm(fem.vertex_gradient(m, s.X, z, s.dt)[m.free])
    g = fem.vertex_gradient(m, xg, z, s.dt)
    r = np.linalg.norm(g[m.free]) / g0
    assert r <= 2e-4, r
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, cub, 1e-10, 3000)
    H = fem.global_hessian(m, xg, s.dt)
    pred = np.linalg.norm(np.linalg.solve(H, fem.free_vector(m, g)))
    err = np.linalg.norm((xg - o.x)[m.free])
    assert err <= 2.0 * pred + 1e-7 * np.linalg.norm(o.x - s.X), (err, pred)
    assert rel(v.cpu().numpy(), (xg - s.X) / s.dt, v.cpu().numpy()) <= 1e-6


def test_step_host_api_matches_device_api(cuda, cube):
    s, m, cub = cube
    gm = gpu_mesh(s, cub)
    xh = s.X.copy()
    vh = s.v0.copy()
    r1 = gm.step_host(xh, vh, p.step_opts(precision=p.FP64))
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    r2 = gm.step(x, v, p.step_opts(precision=p.FP64))
    assert r1.sweeps == r2.sweeps
    assert np.array_equal(xh, x.cpu().numpy()) and np.array_equal(vh, v.cpu().numpy())


def test_import_export_roundtrip(cuda, beam):
    s, m, cub = beam
    gm = gpu_mesh(s, cub)
    e, w, u, _ = gm.precompute_export()
    assert np.array_equal(e, cub.elem)
    assert np.array_equal(w, cub.weight)
    assert np.array_equal(u, cub.ubar)


def test_not_precomputed_is_reported(cuda, cube):
    s, m, _ = cube
    gm = gpu_mesh(s)
    with pytest.raises(p.JGS2Error) as ei:
        gm.step(t(s.X, cuda), t(s.v0, cuda), p.step_opts())
    assert ei.value.status == 4
    # uncorrected Jacobi needs no precompute
    gm.step(t(s.X, cuda), t(s.v0, cuda), p.step_opts(correction=p.CORR_OFF, max_sweeps=3))


def _sampled_direction_check(cuda, s, prec, n_samples, seed):
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=seed, w_max=0.5, u_sigma=0.2)
    gm = gpu_mesh(s, precompute.Cubature(elem, w, u, np.zeros(len(s.X))))
    xk = scenes.perturbed_state(s.X, s.pinned, 1e-5, seed=seed + 1)
    v = scenes.perturbed_state(np.zeros_like(s.X), s.pinned, 0.05, seed=seed + 2)
    xg = t(xk, cuda)
    gm.sweeps(t(s.X, cuda), t(v, cuda), xg, 1, p.step_opts(precision=prec, line_search=0))
    D_gpu = xg.cpu().numpy() - xk
    lm = local.LocalMesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    z = fem.inertia_target(s.X, v, s.dt, s.gravity)
    rng = np.random.default_rng(seed)
    free = np.nonzero(~s.pinned.astype(bool))[0]
    for i in rng.choice(free, size=n_samples, replace=False):
        d, _ = lm.direction(i, xk, z, s.dt, elem[i], w[i], u[i])
        assert np.linalg.norm(D_gpu[i] - d) <= TOL[prec] * np.linalg.norm(d), i


@pytest.mark.parametrize("prec", [p.FP32, p.FP64])
def test_full_size_beam_sampled(cuda, prec):
    """The 20x20x100-vertex stiff beam (214,434 tets) in the bench's launch configuration;
    32 sampled vertices checked against the per-vertex oracle."""
    _sampled_direction_check(cuda, scenes.beam_scene(), prec, 32, seed=10)


def test_full_size_spheres_sampled(cuda):
    """The ten-sphere scene (3.47M tets), FP32: 24 sampled vertices against the oracle."""
    _sampled_direction_check(cuda, scenes.spheres_scene(contact=0), p.FP32, 24, seed=20)
