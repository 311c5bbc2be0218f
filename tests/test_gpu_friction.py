"""GPU parity of the wall friction (lagged at the step start; IPC's friction potential on the
vertex-wall pairs) against the oracle, whose friction tests/test_oracle_friction.py pins:
energy and gradient, sweeps (FP64 1e-9, FP32 1e-4 per vertex), and a whole FP64 step, for
the barrier and the penalty forms. The friction changes each result (checked against the
frictionless oracle)."""
import dataclasses

import numpy as np
import pytest

import paper_2506_06494_b300 as p
import scenes
from oracle import fem, precompute, sweep

pytestmark = pytest.mark.gpu

TOL = {p.FP64: 1e-9, p.FP32: 1e-4}
MU, EPS_V = 0.3, 1e-3


def t(a, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def omesh(s, mu=MU):
    m = fem.Mesh(s.X, s.tets, s.youngs, s.poisson, s.density, s.pinned)
    return m.enable_contact(s.planes, s.dhat, s.kappa, use_penalty=s.contact == 2, friction_mu=mu,
                            friction_eps_v=EPS_V)


def slid_state(s, seed):
    """Positions after part of a step's slide, plus noise: tangential slips on both sides of
    the smoothing slip eps_v h."""
    r = np.random.default_rng(seed)
    x = s.X + s.v0 * s.dt * 0.3
    return x + r.normal(0.0, 3e-6, x.shape)


@pytest.mark.parametrize("form", [1, 2])
def test_energy_gradient_with_friction(cuda, form):
    s = dataclasses.replace(scenes.slide_scene(), contact=form)
    m = omesh(s)
    m.contact.lag_friction(s.X, s.dt)
    assert np.count_nonzero(m.contact.fr[1]) >= 4
    x = slid_state(s, 1)
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    g = p.Mesh.from_scene(s, friction_mu=MU, friction_eps_v=EPS_V)
    E, gr = g.energy_gradient(t(s.X, cuda), t(s.v0, cuda), t(x, cuda))
    go = fem.vertex_gradient(m, x, z, s.dt)
    assert np.abs(gr.cpu().numpy() - go).max() <= 1e-10 * np.abs(go).max()
    assert abs(E - fem.energy(m, x, z, s.dt)) <= 1e-10 * abs(E)
    # friction is in both
    gf, _ = m.contact.friction_terms(x, m.V)
    assert np.abs(gf).max() > 1e-3 * np.abs(go).max()


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
@pytest.mark.parametrize("corr", [p.CORR_ASM, p.CORR_OFF])
@pytest.mark.parametrize("form", [1, 2])
def test_sweeps_with_friction(cuda, prec, corr, form):
    s = dataclasses.replace(scenes.slide_scene(), contact=form)
    m = omesh(s)
    m.contact.lag_friction(s.X, s.dt)
    x = slid_state(s, 2)
    elem, w, u = scenes.random_cubature(s.X, s.tets, s.pinned, 4, seed=4, w_max=0.3, u_sigma=0.1)
    cub = None if corr == p.CORR_OFF else precompute.Cubature(elem, w, u, np.zeros(len(s.X)))
    g = p.Mesh.from_scene(s, friction_mu=MU, friction_eps_v=EPS_V)
    g.precompute_import(elem, w, u)
    xg = t(x, cuda)
    g.sweeps(t(s.X, cuda), t(s.v0, cuda), xg, 2, p.step_opts(precision=prec, correction=corr))
    z = fem.inertia_target(s.X, s.v0, s.dt, s.gravity)
    xo = sweep.run_sweeps(m, x, z, s.dt, cub, 2)
    disp = np.linalg.norm(xo - x, axis=1).max()
    err = np.linalg.norm(xg.cpu().numpy() - xo, axis=1).max() / disp
    assert err <= TOL[prec], err
    m0 = omesh(s, mu=0.0)
    x0 = sweep.run_sweeps(m0, x, z, s.dt, cub, 2)
    assert np.linalg.norm(x0 - xo, axis=1).max() > 1e3 * TOL[p.FP64] * disp


@pytest.mark.parametrize("form", [1, 2])
def test_step_with_friction_fp64_matches_oracle(cuda, form):
    s = dataclasses.replace(scenes.slide_scene(), contact=form)
    m = omesh(s)
    g = p.Mesh.from_scene(s, friction_mu=MU, friction_eps_v=EPS_V)
    x = t(s.X, cuda)
    v = t(s.v0, cuda)
    rep = g.step(x, v, p.step_opts(precision=p.FP64, correction=p.CORR_OFF, max_sweeps=80, record_trace=1))
    o = sweep.step(m, s.X, s.v0, s.dt, s.gravity, None, 1e-4, 80)
    assert rep.sweeps == o.sweeps
    tr = np.array(rep.trace[:rep.trace_len])
    assert np.allclose(tr, o.residuals, rtol=1e-6, atol=1e-12)
    assert np.linalg.norm(x.cpu().numpy() - o.x) / np.linalg.norm(o.x - s.X) <= 1e-9
    o0 = sweep.step(omesh(s, mu=0.0), s.X, s.v0, s.dt, s.gravity, None, 1e-4, 80)
    assert np.linalg.norm(o0.x - o.x) > 1e-6 * np.linalg.norm(o.x - s.X)
