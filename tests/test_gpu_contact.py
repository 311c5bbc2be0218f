"""GPU parity of the contact path (Sec. 7) against the oracle's brute-force contact: the IPC
barrier (contact = 1) and the implicit quadratic penalty (contact = 2).

Pair lists must match bit-exactly (canonical rows); energies, gradients and sweeps to the
FP64 / FP32 tolerances of the sweep tests (per vertex).
"""
import dataclasses

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute, sweep

pytestmark = pytest.mark.gpu

TOL = {p.FP64: 1e-9, p.FP32: 1e-4}


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def omesh(s):
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return m.enable_contact(s.planes, s.dhat, s.kappa, use_penalty=s.contact == 2)


def near_contact_state(s, seed):
    """The scene advanced by its initial velocity until its gaps are about a third of dhat
    (drop: 0.5 mm floor gap; stack: 1.5 mm between the blocks), plus noise."""
    x = s.X + s.v0 * (0.0012 if s.name == "drop" else 0.004)
    r = np.random.default_rng(seed)
    return x + r.normal(0.0, 1e-5, x.shape) * (~s.pinned.astype(bool))[:, None]


@pytest.mark.parametrize("radius", [1e-3, 2e-3, 5e-3])
def test_pair_list_bit_exact(cuda, radius):
    s = scenes.stack_scene()
    m = omesh(s)
    x = near_contact_state(s, 1)
    ref = m.contact.canonical(m.contact.pairs(x, radius))
    g = p.Mesh.from_scene(s)
    got = g.contact_pairs(t(s.X, cuda), t(x, cuda), radius)
    assert [tuple(r) for r in got] == [tuple(r) for r in ref]
    kinds = {r[0] for r in ref}
    assert kinds == {0, 1, 2} or radius < 2e-3


@pytest.mark.parametrize("form", [1, 2])
def test_energy_gradient_with_contact(cuda, form):
    s = dataclasses.replace(scenes.stack_scene(), contact=form)
    m = omesh(s)
    x = near_contact_state(s, 2)
    assert len(m.contact.pairs(x, s.dhat)) > 0
    g = p.Mesh.from_scene(s)
    E, gr = g.energy_gradient(t(s.X, cuda), t(s.v0, cuda), t(x, cuda))
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    go = fem.vertex_gradient(m, x, z, s.dt)
    assert np.abs(gr.cpu().numpy() - go).max() <= 1e-10 * np.abs(go).max()
    assert abs(E - fem.energy(m, x, z, s.dt)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
@pytest.mark.parametrize("corr", [p.CORR_ASM, p.CORR_OFF])
@pytest.mark.parametrize("name", ["drop", "stack"])
@pytest.mark.parametrize("form", [1, 2])
def test_sweeps_with_contact(cuda, prec, corr, name, form):
    s = scenes.drop_scene(nv=3) if name == "drop" else scenes.stack_scene()
    s = dataclasses.replace(s, contact=form)
    m = omesh(s)
    x = near_contact_state(s, 3)
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=4, w_max=0.3, u_sigma=0.1)
    cub = precompute.Cubature(elem, w, u, np.zeros(len(s.X)))
    g = p.Mesh.from_scene(s)
    g.precompute_import(elem, w, u)
    xg = t(x, cuda)
    g.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 2, p.step_opts(precision=prec, correction=corr))
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    xo = sweep.run_sweeps(m, x, z, s.dt, None if corr == p.CORR_OFF else cub, 2)
    # per vertex: largest vertex error over the largest vertex displacement
    err = np.linalg.norm(xg.cpu().numpy() - xo, axis=1).max() / np.linalg.norm(xo - x, axis=1).max()
    assert err <= TOL[prec], err


@pytest.mark.parametrize("form", [1, 2])
def test_step_with_contact_fp64_matches_oracle(cuda, form):
    s = dataclasses.replace(scenes.drop_scene(nv=3), contact=form)
    m = omesh(s)
    g = p.Mesh.from_scene(s)
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    rep = g.step(x, v, p.step_opts(precision=p.FP64, correction=p.CORR_OFF, max_sweeps=60, record_trace=1))
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 60)
    assert rep.sweeps == o.sweeps
    tr = np.array(rep.trace[:rep.trace_len])
    assert np.allclose(tr, o.residuals, rtol=1e-6, atol=1e-12)
    assert np.linalg.norm(x.cpu().numpy() - o.x) / np.linalg.norm(o.x - s.X) <= 1e-9
    assert x.cpu().numpy()[:, 2].min() > 0.0


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
@pytest.mark.parametrize("form", [1, 2])
def test_contact_aware_coupling_matches_oracle(cuda, prec, form):
    """Sec. 7's two-way coupling (contact_coupling = 1): vertices of the upper block that touch
    the lower block solve their local systems with the lower block's colliding vertices moving
    along; two corrected sweeps against the oracle's coupled sweeps. The coupling changes the
    result (it is compared with the uncoupled sweeps too)."""
    s = dataclasses.replace(scenes.stack_scene(), contact=form)
    m = omesh(s)
    x = near_contact_state(s, 5)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    g0 = fem.vertex_gradient(m, x, z, s.dt)
    assert len(sweep.coupled_local_terms(m, x, g0, fem.vertex_diag_blocks(m, x, s.dt))) > 0
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=4, w_max=0.3, u_sigma=0.1)
    cub = precompute.Cubature(elem, w, u, np.zeros(len(s.X)))
    g = p.Mesh.from_scene(s)
    g.precompute_import(elem, w, u)
    xg = t(x, cuda)
    g.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 2, p.step_opts(precision=prec, contact_coupling=1))
    xo = sweep.run_sweeps(m, x, z, s.dt, cub, 2, coupled=True)
    xu = sweep.run_sweeps(m, x, z, s.dt, cub, 2, coupled=False)
    disp = np.linalg.norm(xo - x, axis=1).max()
    err = np.linalg.norm(xg.cpu().numpy() - xo, axis=1).max() / disp
    assert err <= TOL[prec], err
    assert np.linalg.norm(xu - xo, axis=1).max() > 1e3 * TOL[p.FP64] * disp
